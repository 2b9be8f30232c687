// Host side of libmpm: the context, memory management and the C ABI.
//
// Principles followed (Sec. 3.1): no reallocation once running except the
// 4x-when-half-full growth of the particle and grid containers; the fewest
// kernels per substep (P2G, grid update, G2P); no host/device sync in a
// substep except one wait for the new block count when a rebuild runs.
//
// Rebuild trigger without a per-substep sync: G2P of substep s writes a flag
// word when some particle's stencil, widened by one cell per side, reaches
// an unmapped block.  Particles move less than one cell per substep (the CFL
// condition), so that flag only has to be acted on before the P2G of
// substep s + 2.  mpm_substep(s) therefore waits on the flag of substep
// s - 2, which the GPU has finished while it runs substep s - 1: the host
// never stalls the stream.  A particle that outruns the mapping anyway
// (faster than one cell per substep) is reported as MPM_EDOMAIN, never
// written out of bounds.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "device_math.cuh"
#include "internal.h"

using namespace mpm;

namespace mpm {

// ceilings.cu: the L2 reduction-rate probe (not part of the substep)
cudaError_t launch_debug_red_rate(float4* grid, int64_t nodes, int64_t threads, int reds, int pattern,
                                  cudaStream_t s);
// rebuild.cu: one warp polls an mbarrier no copy completes, with the bounded
// wait of the staged transfer kernels, and sets ST_TIMEOUT when it gives up.
void launch_debug_wait_timeout(int max_iter, uint32_t* err, cudaStream_t s);
}  // namespace mpm

namespace {

constexpr int kRing = 4;

// Status words (dstat on the device, hstat its pinned mirror, same indices):
//   [0]                    sticky error bits
//   [kFlag0 + 2 slot]      flag word of ring slot `slot`; the word after it
//                          holds the substep's max |v|^2 when speeds are tracked
//   [kCountWord]           block count of the last rebuild
//   [kErrCopyWord]         host copy of the error bits
constexpr int kFlag0 = 2;
constexpr int kCountWord = kFlag0 + 2 * kRing;
constexpr int kErrCopyWord = kCountWord + 1;
inline int flag_word(int slot) { return kFlag0 + 2 * slot; }

struct ProfRec {
    int phase;
    cudaEvent_t a, b;
};

}  // namespace

struct mpm_ctx {
    mpm_config cfg{};
    SimParams sp{};
    mpm_allocator alloc{};
    bool have_alloc = false;
    cudaStream_t stream = nullptr;

    // particles (double-buffered so the sort can permute out of place)
    int64_t n = 0, cap = 0;
    void* pbuf[2] = {nullptr, nullptr};
    size_t pbuf_bytes = 0;
    PartView pv[2]{};
    int cur = 0;
    int aosoa = 0;   // particle store layout of both buffers (PartView::aosoa)

    // block table (direct-mapped by Morton code) and physical blocks
    int64_t n_slots = 0;
    int32_t* flags = nullptr;
    int32_t* ranks = nullptr;
    int32_t* table = nullptr;
    int32_t* pslot = nullptr;
    uint8_t* interior = nullptr;   // per physical block, n_slots bytes
    void* scan_scr = nullptr;
    size_t scan_scr_bytes = 0;
    int32_t n_pblocks = 0;
    int64_t grid_cap = 0;
    float4* grid[2] = {nullptr, nullptr};
    float4* gold = nullptr;   // ASFLIP: grid velocity before forces, same layout and capacity
    int gcur = 0;

    // sort
    int64_t sort_cap = 0;
    uint32_t* keys = nullptr;
    int32_t* vals = nullptr;
    uint32_t* skeys = nullptr;
    int32_t* svals = nullptr;
    void* sort_scr = nullptr;
    size_t sort_scr_bytes = 0;
    bool keys_valid = false;

    // staging for host copies and layout changes
    void* stage = nullptr;
    size_t stage_bytes = 0;

    // status words (layout above kFlag0)
    uint32_t* dstat = nullptr;
    uint32_t* hstat = nullptr;  // pinned mirror
    cudaEvent_t ev[kRing] = {};
    int64_t step = 0, last_rebuild = -1, last_resort = -1;
    bool need_rebuild = true;
    // fused G2P2G mode: grid[gcur] holds the momentum of the current state
    // (primed); the stress channels are stale after fused substeps
    bool primed = false;
    float primed_dt = 0.0f;   // the dt whose stress impulse the primed momentum carries
    bool tau_valid = true;

    int64_t rebuilds = 0, launches = 0;
    std::string err;

    // CUDA-graph replay of the substep (P2G, grid update, G2P, flag copy):
    // one graph per (mode, flag slot, current grid buffer, current particle
    // buffer); every pointer and size a graph captures is fixed until the
    // next rebuild, particle addition or variant change, which drop them
    // all.  A new dt re-captures the substep and updates the instantiated
    // graph in place (same topology, new kernel arguments).
    bool graphs = false;
    cudaGraphExec_t gexec[8 * kRing] = {};   // by mode, flag slot, current grid buffer, current particle buffer
    float gexec_dt[8 * kRing] = {};          // the dt each instantiated graph carries
    int64_t graph_launches = 0;
    int64_t graph_drop_step = -1;   // substep of the last drop: that substep launches directly

    // adaptive dt (mpm_advance): speeds known from the ring (substeps >=
    // speed_ring_from write their max |v|^2) or from a reduction taken at the
    // start of substep known_step; both reset when particles change
    bool track_speed = false;       // each substep also reduces max |v|^2 into its ring slot
    float c_max = 0.0f;             // largest dilatational wave speed of the materials
    int64_t speed_ring_from = -1;
    int64_t known_step = -1;
    float known_v2 = 0.0f;
    float last_dt = 0.0f;

    // host mirror of the block table (refreshed at every rebuild), used to
    // decide on the host whether emitted particles land in mapped blocks
    int32_t* htable = nullptr;
    bool htable_valid = false;
    // pinned staging ring for asynchronous emission
    static constexpr int kEmitSlots = 4;
    float* emit_host[kEmitSlots] = {};
    size_t emit_host_bytes[kEmitSlots] = {};
    float* emit_dev[kEmitSlots] = {};
    size_t emit_dev_bytes[kEmitSlots] = {};
    cudaEvent_t emit_ev[kEmitSlots] = {};
    int emit_next = 0;
    int64_t emitted = 0;

    bool prof = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[MPM_PHASES] = {0, 0, 0, 0};
    int64_t prof_launch[MPM_PHASES] = {0, 0, 0, 0};
};

namespace {

mpm_status fail(mpm_ctx* c, mpm_status st, const char* msg)
{
    if (c)
        c->err = msg;
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                              \
            return MPM_ECUDA;                                                                           \
        }                                                                                               \
    } while (0)

void* dalloc(mpm_ctx* ctx, size_t bytes)
{
    if (bytes == 0)
        bytes = 256;
    if (ctx->have_alloc)
        return ctx->alloc.alloc(bytes, (void*)ctx->stream, ctx->alloc.user);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess)
        return nullptr;
    return p;
}

void dfree(mpm_ctx* ctx, void* p, size_t bytes)
{
    if (!p)
        return;
    if (bytes == 0)
        bytes = 256;
    if (ctx->have_alloc)
        ctx->alloc.free(p, bytes, (void*)ctx->stream, ctx->alloc.user);
    else
        cudaFreeAsync(p, ctx->stream);
}

template <class T>
mpm_status realloc_buf(mpm_ctx* ctx, T*& p, size_t& have, size_t want)
{
    if (want <= have && p)
        return MPM_OK;
    dfree(ctx, (void*)p, have);
    p = (T*)dalloc(ctx, want);
    have = p ? want : 0;
    return p ? MPM_OK : fail(ctx, MPM_ENOMEM, "device allocation failed");
}

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// The float store sized for either layout (AoSoA packets carry one unused
// line each), then the ids and the material bytes.
size_t store_bytes(int64_t cap) { return (size_t)(cap / 32) * kPacketFloats * 4; }
size_t part_bytes(int64_t cap) { return store_bytes(cap) + (size_t)cap * (1 + 4) + 512; }

PartView make_view(void* base, int64_t cap, int aosoa)
{
    PartView v;
    v.soa = (float*)base;
    v.cap = cap;
    v.aosoa = aosoa;
    char* p = (char*)base + store_bytes(cap);
    v.id = (int32_t*)p;
    v.mat = (uint8_t*)(p + (size_t)cap * 4);
    return v;
}

// Phase timing helpers (events on the context's stream).
void prof_begin(mpm_ctx* ctx, cudaEvent_t& a)
{
    if (!ctx->prof)
        return;
    if (ctx->ev_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        a = e;
    } else {
        a = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
    }
    cudaEventRecord(a, ctx->stream);
}

void prof_drain(mpm_ctx* ctx, size_t keep)
{
    while (ctx->prof_recs.size() > keep) {
        ProfRec r = ctx->prof_recs.front();
        ctx->prof_recs.erase(ctx->prof_recs.begin());
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        ctx->prof_ms[r.phase] += ms;
        ctx->prof_launch[r.phase] += 1;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
}

void prof_end(mpm_ctx* ctx, int phase, cudaEvent_t a)
{
    if (!ctx->prof)
        return;
    cudaEvent_t b;
    prof_begin(ctx, b);
    ctx->prof_recs.push_back({phase, a, b});
    if (ctx->prof_recs.size() > 4096)
        prof_drain(ctx, 2048);
}

mpm_status device_error(mpm_ctx* ctx)
{
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&ctx->hstat[kErrCopyWord], ctx->dstat, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    e = ctx->hstat[kErrCopyWord];
    if (e & ST_ENONFINITE)
        return fail(ctx, MPM_ENONFINITE, "a particle position became non-finite");
    if (e & ST_EDOMAIN)
        return fail(ctx, MPM_EDOMAIN, "a particle stencil left the grid");
    if (e & ST_MISSED)
        return fail(ctx, MPM_EDOMAIN, "a particle outran its mapped blocks (moved more than one cell per substep)");
    if (e & ST_TIMEOUT)
        return fail(ctx, MPM_ETIMEOUT, "an asynchronous copy into shared memory did not complete in time");
    return MPM_OK;
}

mpm_status ensure_particle_capacity(mpm_ctx* ctx, int64_t need)
{
    if (ctx->cfg.max_particles > 0 && need > ctx->cfg.max_particles)
        return fail(ctx, MPM_ECAPACITY, "max_particles exceeded");
    if (ctx->pbuf[0] && (need <= ctx->cap / 2 ||
                         (ctx->cfg.max_particles > 0 && ctx->cap >= ctx->cfg.max_particles && need <= ctx->cap)))
        return MPM_OK;
    // Sec. 3.1: grow to 4x the requested size once more than half full.
    int64_t ncap = round_up(4 * need, kCapQuantum);
    if (ctx->cfg.max_particles > 0 && ncap > ctx->cfg.max_particles)
        ncap = round_up(ctx->cfg.max_particles, kCapQuantum);
    if (ncap > (int64_t)0x7fffff00)
        return fail(ctx, MPM_ECAPACITY, "particle count exceeds 2^31");
    size_t nb = part_bytes(ncap);
    void* nbuf[2] = {dalloc(ctx, nb), dalloc(ctx, nb)};
    if (!nbuf[0] || !nbuf[1]) {
        dfree(ctx, nbuf[0], nb);
        dfree(ctx, nbuf[1], nb);
        return fail(ctx, MPM_ENOMEM, "particle allocation failed");
    }
    PartView nv = make_view(nbuf[0], ncap, ctx->aosoa);
    if (ctx->n > 0) {
        const PartView& ov = ctx->pv[ctx->cur];
        if (ctx->aosoa)   // whole packets: their layout does not depend on the capacity
            CK(cudaMemcpyAsync(nv.soa, ov.soa, (size_t)((ctx->n + 31) / 32) * kPacketFloats * 4,
                               cudaMemcpyDeviceToDevice, ctx->stream));
        else
            for (int c = 0; c < kChannels; ++c)
                CK(cudaMemcpyAsync(nv.ch(c), ov.ch(c), (size_t)ctx->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(nv.id, ov.id, (size_t)ctx->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(nv.mat, ov.mat, (size_t)ctx->n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    dfree(ctx, ctx->pbuf[0], ctx->pbuf_bytes);
    dfree(ctx, ctx->pbuf[1], ctx->pbuf_bytes);
    ctx->pbuf[0] = nbuf[0];
    ctx->pbuf[1] = nbuf[1];
    ctx->pbuf_bytes = nb;
    ctx->pv[0] = nv;
    ctx->pv[1] = make_view(nbuf[1], ncap, ctx->aosoa);
    ctx->cur = 0;
    ctx->cap = ncap;
    // sort buffers follow the particle capacity
    size_t kb = (size_t)ncap * 4, have;
    have = ctx->sort_cap * 4;
    mpm_status st;
    size_t h1 = have, h2 = have, h3 = have, h4 = have;
    if ((st = realloc_buf(ctx, ctx->keys, h1, kb)) != MPM_OK) return st;
    if ((st = realloc_buf(ctx, ctx->vals, h2, kb)) != MPM_OK) return st;
    if ((st = realloc_buf(ctx, ctx->skeys, h3, kb)) != MPM_OK) return st;
    if ((st = realloc_buf(ctx, ctx->svals, h4, kb)) != MPM_OK) return st;
    ctx->sort_cap = ncap;
    if ((st = realloc_buf(ctx, ctx->sort_scr, ctx->sort_scr_bytes, radix_sort_scratch_bytes(ncap))) != MPM_OK)
        return st;
    ctx->keys_valid = false;
    return MPM_OK;
}

mpm_status ensure_stage(mpm_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->stage_bytes && ctx->stage)
        return MPM_OK;
    size_t want = bytes < 2 * ctx->stage_bytes ? 2 * ctx->stage_bytes : bytes;
    return realloc_buf(ctx, ctx->stage, ctx->stage_bytes, want);
}

GridView grid_view(mpm_ctx* ctx)
{
    GridView g;
    g.cur = ctx->grid[ctx->gcur];
    g.nxt = ctx->grid[1 - ctx->gcur];
    g.table = ctx->table;
    g.pslot = ctx->pslot;
    g.interior = ctx->interior;
    g.old = ctx->cfg.transfer == MPM_ASFLIP ? ctx->gold : nullptr;
    g.slot = nullptr;
    g.n_pblocks = ctx->n_pblocks;
    return g;
}

// Particle velocities changed outside G2P: the speeds the ring holds no
// longer bound them.
void forget_speeds(mpm_ctx* ctx)
{
    ctx->speed_ring_from = -1;
    ctx->known_step = -1;
}

// The grid update clears the substep's two status words before G2P sets
// them (one launch fewer per substep); without blocks to update, a memset.
void clear_slot(mpm_ctx* ctx, GridView& gv, int slot)
{
    if (gv.n_pblocks > 0)
        gv.slot = &ctx->dstat[flag_word(slot)];
    else
        cudaMemsetAsync(&ctx->dstat[flag_word(slot)], 0, 8, ctx->stream);
}

// One separate substep on the context's stream: clear the flag slot, P2G,
// grid update, G2P, copy the flags to the pinned ring.
void enqueue_separate(mpm_ctx* ctx, float dt, int slot)
{
    cudaStream_t s = ctx->stream;
    GridView gv = grid_view(ctx);
    clear_slot(ctx, gv, slot);
    const PartView& pv = ctx->pv[ctx->cur];
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    prof_begin(ctx, e0);
    launch_p2g(ctx->sp, pv, gv, ctx->n, dt, ctx->dstat, ctx->cfg.p2g_variant, s);
    prof_end(ctx, 1, e0);
    prof_begin(ctx, e1);
    launch_grid_update(ctx->sp, gv, dt, s);
    prof_end(ctx, 2, e1);
    prof_begin(ctx, e2);
    launch_g2p(ctx->sp, pv, gv, ctx->n, dt, &ctx->dstat[flag_word(slot)], ctx->dstat, ctx->cfg.g2p_variant, s);
    prof_end(ctx, 3, e2);
    if (ctx->track_speed)
        launch_max_speed2(pv, ctx->n, &ctx->dstat[flag_word(slot) + 1], s);
    cudaMemcpyAsync(&ctx->hstat[flag_word(slot)], &ctx->dstat[flag_word(slot)], 8, cudaMemcpyDeviceToHost, s);
}

void drop_graphs(mpm_ctx* ctx)
{
    // a context that keeps changing (emission every substep) would capture a
    // graph per substep: the substep of a drop launches directly instead
    ctx->graph_drop_step = ctx->step;
    for (auto& g : ctx->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Rebuild-mapping + full sort (Sec. 4.2.1, Sec. 4.2.2).
mpm_status rebuild(mpm_ctx* ctx)
{
    TraceRange trace("rebuild");
    drop_graphs(ctx);
    cudaEvent_t pa = nullptr;
    prof_begin(ctx, pa);
    cudaStream_t s = ctx->stream;
    int64_t n = ctx->n;
    const SimParams& sp = ctx->sp;
    const bool sort = !ctx->cfg.no_sort;
    if (n > 0) {
        launch_keys(sp, ctx->pv[ctx->cur], n, ctx->keys, ctx->vals, ctx->dstat, s);
        ctx->launches += 1;
        if (sort)
            CK(radix_sort_pairs(ctx->keys, ctx->vals, ctx->skeys, ctx->svals, n, 3 * sp.L + 6, ctx->sort_scr, s,
                                &ctx->launches));
    }
    CK(cudaMemsetAsync(ctx->flags, 0, (size_t)ctx->n_slots * 4, s));
    launch_mark_pblocks(sort ? ctx->skeys : ctx->keys, n, sp.L, ctx->flags, s);
    CK(exclusive_scan(ctx->flags, ctx->ranks, ctx->n_slots, ctx->scan_scr, s, &ctx->launches));
    launch_build_table(ctx->flags, ctx->ranks, ctx->n_slots, ctx->table, ctx->pslot,
                       (int32_t*)&ctx->dstat[kCountWord], s);
    ctx->launches += 2;
    if (n > 0 && sort) {
        launch_permute(ctx->pv[ctx->cur], ctx->pv[1 - ctx->cur], ctx->svals, n, s);
        ctx->launches += 1;
        ctx->cur = 1 - ctx->cur;
    }
    CK(cudaMemcpyAsync(&ctx->hstat[kCountWord], &ctx->dstat[kCountWord], 4, cudaMemcpyDeviceToHost, s));
    if (ctx->htable) {
        CK(cudaMemcpyAsync(ctx->htable, ctx->table, (size_t)ctx->n_slots * 4, cudaMemcpyDeviceToHost, s));
        ctx->htable_valid = true;
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    int32_t npb = (int32_t)ctx->hstat[kCountWord];
    ctx->n_pblocks = npb;
    launch_interior(sp, ctx->table, ctx->pslot, npb, ctx->interior, s);
    ctx->launches += 1;
    if ((int64_t)npb > ctx->grid_cap / 2 || !ctx->grid[0]) {
        int64_t gcap = 4 * (int64_t)npb;
        if (gcap > ctx->n_slots)
            gcap = ctx->n_slots;
        if (gcap < 64)
            gcap = 64;
        size_t have0 = (size_t)ctx->grid_cap * 1024, have1 = have0;
        mpm_status st;
        if ((st = realloc_buf(ctx, ctx->grid[0], have0, (size_t)gcap * 1024)) != MPM_OK) return st;
        if ((st = realloc_buf(ctx, ctx->grid[1], have1, (size_t)gcap * 1024)) != MPM_OK) return st;
        if (ctx->cfg.transfer == MPM_ASFLIP) {
            size_t have2 = (size_t)ctx->grid_cap * 1024;
            if ((st = realloc_buf(ctx, ctx->gold, have2, (size_t)gcap * 1024)) != MPM_OK) return st;
        }
        ctx->grid_cap = gcap;
    }
    if (npb > 0) {
        CK(cudaMemsetAsync(ctx->grid[0], 0, (size_t)npb * 1024, s));
        CK(cudaMemsetAsync(ctx->grid[1], 0, (size_t)npb * 1024, s));
    }
    ctx->gcur = 0;
    ctx->primed = false;
    ctx->keys_valid = sort;
    ctx->need_rebuild = false;
    ctx->last_rebuild = ctx->step;
    ctx->rebuilds += 1;
    prof_end(ctx, 0, pa);
    return MPM_OK;
}

bool valid_material(const mpm_material& m)
{
    if (m.kind < MPM_ELASTIC || m.kind > MPM_NHSAND)
        return false;
    if (m.kind == MPM_NACC && !(m.friction_M > 0.f && m.cohesion >= 0.f && m.hardening >= 0.f))
        return false;
    if (!(m.rho > 0.f) || !(m.E > 0.f))
        return false;
    if (m.kind != MPM_FLUID && !(m.nu > -1.f && m.nu < 0.5f))
        return false;
    if (m.kind == MPM_SNOW && !(m.theta_c >= 0.f && m.theta_c < 1.f && m.theta_s >= 0.f))
        return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

mpm_status mpm_create(const mpm_config* cfg, const mpm_material* mats, int n_mats, const mpm_allocator* allocator,
                      void* cuda_stream, mpm_ctx** out)
{
    if (!cfg || !out || !mats || n_mats < 1 || n_mats > kMaxMaterials)
        return MPM_EINVAL;
    *out = nullptr;
    if (!(cfg->dx > 0.f) || cfg->wall < 0 || (cfg->boundary != MPM_STICKY && cfg->boundary != MPM_SLIP))
        return MPM_EINVAL;
    int maxres = 0;
    for (int a = 0; a < 3; ++a) {
        if (cfg->res[a] < 8 || cfg->res[a] > 1024)
            return MPM_EINVAL;
        maxres = cfg->res[a] > maxres ? cfg->res[a] : maxres;
    }
    if (cfg->use_g2p2g != 0 && cfg->use_g2p2g != 1)
        return MPM_EINVAL;
    if (cfg->no_sort != 0 && cfg->no_sort != 1)
        return MPM_EINVAL;
    if (cfg->resort_interval < 0)
        return MPM_EINVAL;
    if (cfg->transfer != MPM_APIC && cfg->transfer != MPM_ASFLIP)
        return MPM_EINVAL;
    if (cfg->transfer == MPM_ASFLIP) {
        const float w[3] = {cfg->flip_alpha, cfg->flip_beta_min, cfg->flip_beta_max};
        for (float v : w)
            if (!(v >= 0.f && v <= 1.f))
                return MPM_EINVAL;
        if (!(cfg->flip_compress_margin >= 0.f && cfg->flip_compress_margin < 1.f))
            return MPM_EINVAL;
        if (cfg->use_g2p2g)
            return MPM_EINVAL;   // the fused transfer has no ASFLIP form
    }
    if (cfg->p2g_variant < 0 || cfg->p2g_variant >= kP2GVariants)
        return MPM_EINVAL;
    if (cfg->g2p_variant < 0 || cfg->g2p_variant >= kG2PVariants)
        return MPM_EINVAL;
    for (int i = 0; i < n_mats; ++i)
        if (!valid_material(mats[i]))
            return MPM_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free))
        return MPM_EINVAL;
    mpm_ctx* ctx = new (std::nothrow) mpm_ctx();
    if (!ctx)
        return MPM_ENOMEM;
    ctx->cfg = *cfg;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        ctx->alloc = *allocator;
        ctx->have_alloc = true;
    }
    SimParams& sp = ctx->sp;
    for (int a = 0; a < 3; ++a) {
        sp.res[a] = cfg->res[a];
        sp.g[a] = cfg->gravity[a];
    }
    sp.dx = cfg->dx;
    sp.inv_dx = 1.0f / cfg->dx;
    sp.boundary = cfg->boundary;
    sp.wall = cfg->wall;
    sp.transfer = cfg->transfer;
    sp.flip_alpha = cfg->transfer == MPM_ASFLIP ? cfg->flip_alpha : 0.f;
    sp.flip_beta_min = cfg->transfer == MPM_ASFLIP ? cfg->flip_beta_min : 0.f;
    sp.flip_beta_max = cfg->transfer == MPM_ASFLIP ? cfg->flip_beta_max : 0.f;
    sp.flip_margin = cfg->transfer == MPM_ASFLIP ? cfg->flip_compress_margin : 0.f;
    sp.cta_warps = 4;
    int L = 0;
    while ((4 << L) < maxres)
        ++L;
    sp.L = L;
    sp.n_mats = n_mats;
    for (int i = 0; i < n_mats; ++i) {
        sp.mat[i] = make_mat_params(mats[i]);
        const MatParams& m = sp.mat[i];
        // dilatational (p-wave) speed: sqrt((lambda + 2 mu) / rho); for the
        // fluid the bulk modulus of p = K (J^-gamma - 1) at J = 1 is K gamma
        const double mod = m.kind == MPM_FLUID ? (double)m.K * m.gamma : (double)m.la + 2.0 * m.mu;
        const double c = sqrt(mod > 0.0 ? mod / m.rho : 0.0);
        if (c > ctx->c_max)
            ctx->c_max = (float)c;
    }
    ctx->n_slots = (int64_t)1 << (3 * L);

    mpm_status st = MPM_OK;
    size_t b0 = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0, b5 = 0;
    size_t sb = (size_t)ctx->n_slots * 4;
    if ((st = realloc_buf(ctx, ctx->flags, b0, sb)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->ranks, b1, sb)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->table, b2, sb)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->pslot, b3, sb)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->interior, b5, (size_t)ctx->n_slots)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->dstat, b4, 256)) != MPM_OK ||
        (st = realloc_buf(ctx, ctx->scan_scr, ctx->scan_scr_bytes, scan_scratch_bytes(ctx->n_slots))) != MPM_OK) {
        mpm_destroy(ctx);
        return st;
    }
    if (cudaMallocHost(&ctx->hstat, 256) != cudaSuccess) {
        ctx->hstat = nullptr;
        mpm_destroy(ctx);
        return MPM_ENOMEM;
    }
    memset(ctx->hstat, 0, 256);
    if (cudaMallocHost(&ctx->htable, (size_t)ctx->n_slots * 4) != cudaSuccess) {
        ctx->htable = nullptr;
        mpm_destroy(ctx);
        return MPM_ENOMEM;
    }
    for (int i = 0; i < mpm_ctx::kEmitSlots; ++i)
        if (cudaEventCreateWithFlags(&ctx->emit_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            mpm_destroy(ctx);
            return MPM_ECUDA;
        }
    for (int i = 0; i < kRing; ++i)
        if (cudaEventCreateWithFlags(&ctx->ev[i], cudaEventDisableTiming) != cudaSuccess) {
            mpm_destroy(ctx);
            return MPM_ECUDA;
        }
    if (cudaMemsetAsync(ctx->dstat, 0, 256, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->table, 0xff, sb, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        mpm_destroy(ctx);
        return MPM_ECUDA;
    }
    *out = ctx;
    return MPM_OK;
}

mpm_status mpm_use_graphs(mpm_ctx* ctx, int on)
{
    if (!ctx || (on != 0 && on != 1))
        return MPM_EINVAL;
    if (on && ctx->stream == nullptr)
        return fail(ctx, MPM_EINVAL, "CUDA graphs need a stream other than the legacy default stream");
    if (!on)
        drop_graphs(ctx);
    ctx->graphs = on != 0;
    return MPM_OK;
}

int64_t mpm_graph_launches(const mpm_ctx* ctx)
{
    return ctx ? ctx->graph_launches : 0;
}

void mpm_destroy(mpm_ctx* ctx)
{
    if (!ctx)
        return;
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    for (auto& r : ctx->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->ev_pool)
        cudaEventDestroy(e);
    size_t sb = (size_t)ctx->n_slots * 4;
    dfree(ctx, ctx->pbuf[0], ctx->pbuf_bytes);
    dfree(ctx, ctx->pbuf[1], ctx->pbuf_bytes);
    dfree(ctx, ctx->flags, sb);
    dfree(ctx, ctx->ranks, sb);
    dfree(ctx, ctx->table, sb);
    dfree(ctx, ctx->pslot, sb);
    dfree(ctx, ctx->interior, (size_t)ctx->n_slots);
    dfree(ctx, ctx->scan_scr, ctx->scan_scr_bytes);
    dfree(ctx, ctx->grid[0], (size_t)ctx->grid_cap * 1024);
    dfree(ctx, ctx->grid[1], (size_t)ctx->grid_cap * 1024);
    dfree(ctx, ctx->gold, (size_t)ctx->grid_cap * 1024);
    size_t kb = (size_t)ctx->sort_cap * 4;
    dfree(ctx, ctx->keys, kb);
    dfree(ctx, ctx->vals, kb);
    dfree(ctx, ctx->skeys, kb);
    dfree(ctx, ctx->svals, kb);
    dfree(ctx, ctx->sort_scr, ctx->sort_scr_bytes);
    dfree(ctx, ctx->stage, ctx->stage_bytes);
    dfree(ctx, ctx->dstat, 256);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->hstat)
        cudaFreeHost(ctx->hstat);
    if (ctx->htable)
        cudaFreeHost(ctx->htable);
    for (int i = 0; i < mpm_ctx::kEmitSlots; ++i) {
        if (ctx->emit_host[i])
            cudaFreeHost(ctx->emit_host[i]);
        dfree(ctx, ctx->emit_dev[i], ctx->emit_dev_bytes[i]);
        if (ctx->emit_ev[i])
            cudaEventDestroy(ctx->emit_ev[i]);
    }
    for (int i = 0; i < kRing; ++i)
        if (ctx->ev[i])
            cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

mpm_status mpm_add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v, const float* vol0,
                             int material, int on_device)
{
    TraceRange trace("mpm_add_particles");
    if (!ctx)
        return MPM_EINVAL;
    if (n < 0 || (n > 0 && !x) || material < 0 || material >= ctx->sp.n_mats)
        return fail(ctx, MPM_EINVAL, "mpm_add_particles: bad argument");
    if (n == 0)
        return MPM_OK;
    forget_speeds(ctx);
    mpm_status st = ensure_particle_capacity(ctx, ctx->n + n);
    if (st != MPM_OK)
        return st;
    const float *dx = x, *dv = v, *dvol = vol0;
    if (!on_device) {
        size_t bytes = (size_t)n * 4 * 7 + 1024;
        if ((st = ensure_stage(ctx, bytes)) != MPM_OK)
            return st;
        float* sx = (float*)ctx->stage;
        float* sv = sx + 3 * n;
        float* svol = sv + 3 * n;
        CK(cudaMemcpyAsync(sx, x, (size_t)n * 12, cudaMemcpyHostToDevice, ctx->stream));
        dx = sx;
        if (v) {
            CK(cudaMemcpyAsync(sv, v, (size_t)n * 12, cudaMemcpyHostToDevice, ctx->stream));
            dv = sv;
        }
        if (vol0) {
            CK(cudaMemcpyAsync(svol, vol0, (size_t)n * 4, cudaMemcpyHostToDevice, ctx->stream));
            dvol = svol;
        }
    }
    float dx3 = ctx->sp.dx * ctx->sp.dx * ctx->sp.dx;
    launch_append(ctx->pv[ctx->cur], ctx->n, n, dx, dv, dvol, dx3 / 8.0f, material, ctx->stream);
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    ctx->n += n;
    drop_graphs(ctx);
    ctx->need_rebuild = true;
    ctx->primed = false;
    ctx->keys_valid = false;
    return MPM_OK;
}

// True if every node in [b - margin, b + 2 + margin] per axis (clipped to the
// grid) lies in a block mapped at the last rebuild, by the host mirror.
static bool host_stencil_mapped(const mpm_ctx* ctx, const float* x, int margin)
{
    const SimParams& sp = ctx->sp;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        float X = x[a] * sp.inv_dx - 0.5f;
        if (!(X > -1.0f && X < (float)sp.res[a]))
            return false;
        int b = (int)floorf(X);
        lo[a] = b - margin < 0 ? 0 : b - margin;
        hi[a] = b + 2 + margin > sp.res[a] - 1 ? sp.res[a] - 1 : b + 2 + margin;
        if (b < 0 || b + 2 >= sp.res[a])
            return false;
    }
    for (int z = lo[2] >> 2; z <= hi[2] >> 2; ++z)
        for (int y = lo[1] >> 2; y <= hi[1] >> 2; ++y)
            for (int xx = lo[0] >> 2; xx <= hi[0] >> 2; ++xx)
                if (ctx->htable[morton3((uint32_t)xx, (uint32_t)y, (uint32_t)z)] < 0)
                    return false;
    return true;
}

// Fused G2P2G substep (Sec. 4.1): grid update of the primed momentum, then
// one kernel doing this substep's G2P and the next substep's P2G.  Priming
// (after a rebuild, a state write or an emission) is one plain P2G.
// The steady-state fused substep: clear the flag slot, grid update, G2P2G,
// copy the flags to the pinned ring.
static void enqueue_fused(mpm_ctx* ctx, float dt, int slot)
{
    cudaStream_t s = ctx->stream;
    const PartView& pv = ctx->pv[ctx->cur];
    GridView gv = grid_view(ctx);
    clear_slot(ctx, gv, slot);
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    prof_begin(ctx, e1);
    launch_grid_update(ctx->sp, gv, dt, s);
    prof_end(ctx, 2, e1);
    prof_begin(ctx, e2);
    launch_g2p2g(ctx->sp, pv, gv, ctx->n, dt, &ctx->dstat[flag_word(slot)], ctx->dstat, ctx->cfg.p2g_variant, s);
    prof_end(ctx, 3, e2);
    if (ctx->track_speed)
        launch_max_speed2(pv, ctx->n, &ctx->dstat[flag_word(slot) + 1], s);
    cudaMemcpyAsync(&ctx->hstat[flag_word(slot)], &ctx->dstat[flag_word(slot)], 8, cudaMemcpyDeviceToHost, s);
}

// Replays the steady-state substep of the current mode from its CUDA graph,
// capturing it on first use; graphs are keyed by mode, flag slot, current
// grid buffer and current particle buffer.
static cudaError_t replay(mpm_ctx* ctx, float dt, int slot, bool fused)
{
    cudaStream_t s = ctx->stream;
    const int gi = 16 * (fused ? 1 : 0) + 4 * slot + 2 * ctx->gcur + ctx->cur;
    if (!ctx->gexec[gi] || ctx->gexec_dt[gi] != dt) {
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return e;
        if (fused)
            enqueue_fused(ctx, dt, slot);
        else
            enqueue_separate(ctx, dt, slot);
        e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess)
            return e;
        if (ctx->gexec[gi]) {
            // same nodes, new dt in the kernel arguments: update in place
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(ctx->gexec[gi], graph, &info) != cudaSuccess) {
                cudaGetLastError();   // clear the update's error; instantiate afresh
                cudaGraphExecDestroy(ctx->gexec[gi]);
                ctx->gexec[gi] = nullptr;
            }
        }
        if (!ctx->gexec[gi])
            e = cudaGraphInstantiate(&ctx->gexec[gi], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return e;
        ctx->gexec_dt[gi] = dt;
    }
    ctx->graph_launches += 1;
    return cudaGraphLaunch(ctx->gexec[gi], s);
}

static mpm_status substep_fused(mpm_ctx* ctx, float dt, int slot)
{
    cudaStream_t s = ctx->stream;
    const PartView& pv = ctx->pv[ctx->cur];
    // the primed momentum holds the stress impulse of the dt it was scattered
    // with: a new dt needs a fresh P2G of the current state
    if (ctx->primed && dt != ctx->primed_dt)
        ctx->primed = false;
    if (!ctx->primed) {
        if (!ctx->tau_valid) {
            launch_prepare_stress(ctx->sp, pv, ctx->n, s);
            ctx->launches += 1;
            ctx->tau_valid = true;
        }
        if (ctx->n_pblocks > 0)
            CK(cudaMemsetAsync(ctx->grid[ctx->gcur], 0, (size_t)ctx->n_pblocks * 1024, s));
        cudaEvent_t e0 = nullptr;
        prof_begin(ctx, e0);
        launch_p2g(ctx->sp, pv, grid_view(ctx), ctx->n, dt, ctx->dstat, ctx->cfg.p2g_variant, s);
        prof_end(ctx, 1, e0);
        ctx->launches += 1;
        ctx->primed = true;
    }
    ctx->primed_dt = dt;   // the fused kernel scatters the next substep's momentum with this dt
    if (ctx->graphs && !ctx->prof && ctx->step > ctx->graph_drop_step) {
        CK(replay(ctx, dt, slot, true));
    } else {
        enqueue_fused(ctx, dt, slot);
    }
    ctx->launches += ctx->track_speed ? 3 : 2;
    CK(cudaEventRecord(ctx->ev[slot], s));
    CK(cudaGetLastError());
    ctx->gcur = 1 - ctx->gcur;   // grid[gcur] now holds the momentum of the new state
    ctx->step += 1;
    ctx->tau_valid = false;
    return MPM_OK;
}

mpm_status mpm_emit_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v, const float* vol0,
                              int material, int on_device)
{
    TraceRange trace("mpm_emit_particles");
    if (!ctx)
        return MPM_EINVAL;
    if (n < 0 || (n > 0 && !x) || material < 0 || material >= ctx->sp.n_mats)
        return fail(ctx, MPM_EINVAL, "mpm_emit_particles: bad argument");
    if (n == 0)
        return MPM_OK;
    forget_speeds(ctx);
    if (ctx->n + n > ctx->cap / 2 || !ctx->pbuf[0]) {
        // growth (4x when half full) needs the stream idle; rare by design
        CK(cudaStreamSynchronize(ctx->stream));
        mpm_status st = ensure_particle_capacity(ctx, ctx->n + n);
        if (st != MPM_OK)
            return st;
    }
    const float *dx = x, *dv = v, *dvol = vol0;
    bool mapped = !ctx->need_rebuild && ctx->htable_valid && !on_device;
    if (!on_device) {
        for (int64_t i = 0; i < n && mapped; ++i)
            mapped = host_stencil_mapped(ctx, x + 3 * i, 1);
        int slot = ctx->emit_next;
        ctx->emit_next = (slot + 1) % mpm_ctx::kEmitSlots;
        CK(cudaEventSynchronize(ctx->emit_ev[slot]));   // the slot's previous copy is done
        size_t bytes = (size_t)n * 4 * 7;
        if (bytes > ctx->emit_host_bytes[slot]) {
            if (ctx->emit_host[slot])
                cudaFreeHost(ctx->emit_host[slot]);
            size_t want = bytes * 2;
            if (cudaMallocHost(&ctx->emit_host[slot], want) != cudaSuccess) {
                ctx->emit_host[slot] = nullptr;
                ctx->emit_host_bytes[slot] = 0;
                return fail(ctx, MPM_ENOMEM, "pinned staging allocation failed");
            }
            ctx->emit_host_bytes[slot] = want;
        }
        mpm_status st = realloc_buf(ctx, ctx->emit_dev[slot], ctx->emit_dev_bytes[slot], ctx->emit_host_bytes[slot]);
        if (st != MPM_OK)
            return st;
        float* hx = ctx->emit_host[slot];
        float* hv = hx + 3 * n;
        float* hw = hv + 3 * n;
        memcpy(hx, x, (size_t)n * 12);
        if (v)
            memcpy(hv, v, (size_t)n * 12);
        if (vol0)
            memcpy(hw, vol0, (size_t)n * 4);
        CK(cudaMemcpyAsync(ctx->emit_dev[slot], hx, bytes, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaEventRecord(ctx->emit_ev[slot], ctx->stream));
        dx = ctx->emit_dev[slot];
        dv = v ? dx + 3 * n : nullptr;
        dvol = vol0 ? dx + 6 * n : nullptr;
    }
    float dx3 = ctx->sp.dx * ctx->sp.dx * ctx->sp.dx;
    launch_append(ctx->pv[ctx->cur], ctx->n, n, dx, dv, dvol, dx3 / 8.0f, material, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    ctx->n += n;
    drop_graphs(ctx);
    ctx->emitted += n;
    ctx->keys_valid = false;
    ctx->primed = false;   // the new particles are not in the fused path's momentum
    if (!mapped)
        ctx->need_rebuild = true;
    return MPM_OK;
}

mpm_status mpm_substep(mpm_ctx* ctx, float dt)
{
    TraceRange trace("mpm_substep");
    if (!ctx)
        return MPM_EINVAL;
    if (!(dt > 0.f))
        return fail(ctx, MPM_EINVAL, "mpm_substep: dt must be positive");
    if (ctx->n == 0) {
        ctx->step += 1;
        return MPM_OK;
    }
    // flag of substep step - 2 (see the file comment)
    if (!ctx->need_rebuild && ctx->step >= 2 && ctx->step - 2 >= ctx->last_rebuild) {
        int slot = (int)((ctx->step - 2) % kRing);
        CK(cudaEventSynchronize(ctx->ev[slot]));
        if (ctx->hstat[flag_word(slot)] & (ST_REBUILD_SOFT | ST_REBUILD_HARD))
            ctx->need_rebuild = true;
    }
    if (ctx->need_rebuild) {
        mpm_status st = rebuild(ctx);
        if (st != MPM_OK)
            return st;
    }
    cudaStream_t s = ctx->stream;
    int slot = (int)(ctx->step % kRing);
    const int64_t since = ctx->step - (ctx->last_resort > ctx->last_rebuild ? ctx->last_resort : ctx->last_rebuild);
    if (ctx->cfg.resort_interval > 0 && !ctx->cfg.no_sort && since >= ctx->cfg.resort_interval) {
        launch_resort_window(ctx->sp, ctx->pv[ctx->cur], ctx->pv[1 - ctx->cur], ctx->n, s);
        ctx->cur = 1 - ctx->cur;
        ctx->launches += 1;
        ctx->keys_valid = false;
        ctx->last_resort = ctx->step;
    }
    if (ctx->cfg.use_g2p2g)
        return substep_fused(ctx, dt, slot);
    if (ctx->graphs && !ctx->prof && ctx->step > ctx->graph_drop_step) {
        CK(replay(ctx, dt, slot, false));
    } else {
        enqueue_separate(ctx, dt, slot);
    }
    ctx->launches += ctx->track_speed ? 4 : 3;
    CK(cudaEventRecord(ctx->ev[slot], s));
    CK(cudaGetLastError());
    ctx->gcur = 1 - ctx->gcur;
    ctx->step += 1;
    ctx->tau_valid = true;
    return MPM_OK;
}

mpm_status mpm_advance(mpm_ctx* ctx, double duration, float cfl, float dt_max, int64_t max_substeps, float* dts,
                       int64_t* n_substeps)
{
    TraceRange trace("mpm_advance");
    if (!ctx)
        return MPM_EINVAL;
    if (n_substeps)
        *n_substeps = 0;
    if (!(duration > 0.0) || !(cfl > 0.f && cfl <= 1.f) || !(dt_max > 0.f) || max_substeps < 1)
        return fail(ctx, MPM_EINVAL, "mpm_advance: bad argument");
    if (!ctx->track_speed) {
        ctx->track_speed = true;   // each substep now also reduces the largest speed
        drop_graphs(ctx);
        forget_speeds(ctx);
    }
    const double g = sqrt((double)ctx->sp.g[0] * ctx->sp.g[0] + (double)ctx->sp.g[1] * ctx->sp.g[1] +
                          (double)ctx->sp.g[2] * ctx->sp.g[2]);
    double t = 0.0;
    int64_t k = 0;
    while (duration - t > 1e-9 * duration) {
        if (k >= max_substeps)
            return fail(ctx, MPM_ECAPACITY, "mpm_advance: max_substeps reached before the end of the interval");
        const int64_t s = ctx->step;
        // the freshest speed bound available without stalling the stream:
        // the ring word of substep s - 2 (one substep old at the start of s),
        // else a reduction taken earlier, else a reduction now (one sync)
        float v2 = 0.0f;
        int64_t age = 0;
        if (ctx->n > 0) {
            if (ctx->speed_ring_from >= 0 && s - 2 >= ctx->speed_ring_from) {
                const int slot = (int)((s - 2) % kRing);
                CK(cudaEventSynchronize(ctx->ev[slot]));
                uint32_t bits = ctx->hstat[flag_word(slot) + 1];
                memcpy(&v2, &bits, 4);
                age = 1;
            } else if (ctx->known_step >= 0) {
                v2 = ctx->known_v2;
                age = s - ctx->known_step;
            } else {
                CK(cudaMemsetAsync(&ctx->dstat[kErrCopyWord + 1], 0, 4, ctx->stream));
                launch_max_speed2(ctx->pv[ctx->cur], ctx->n, &ctx->dstat[kErrCopyWord + 1], ctx->stream);
                ctx->launches += 1;
                CK(cudaMemcpyAsync(&ctx->hstat[kErrCopyWord + 1], &ctx->dstat[kErrCopyWord + 1], 4,
                                   cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                uint32_t bits = ctx->hstat[kErrCopyWord + 1];
                memcpy(&v2, &bits, 4);
                ctx->known_v2 = v2;
                ctx->known_step = s;
            }
        }
        if (!(v2 >= 0.0f) || !isfinite(v2))
            return fail(ctx, MPM_ENONFINITE, "mpm_advance: a particle velocity became non-finite");
        const double prev = ctx->last_dt > 0.f ? ctx->last_dt : dt_max;
        const double v_est = sqrt((double)v2) + (double)age * g * prev;
        double dt = (double)cfl * ctx->sp.dx / (v_est + ctx->c_max);
        if (dt > dt_max)
            dt = dt_max;
        const double rem = duration - t;
        if (dt >= rem) {
            dt = rem;
        } else {
            const double parts = ceil(rem / dt);   // equal steps to the end: no sliver
            dt = rem / parts;
        }
        const float dtf = (float)dt;
        mpm_status st = mpm_substep(ctx, dtf);
        if (st != MPM_OK)
            return st;
        if (ctx->speed_ring_from < 0 && ctx->n > 0)
            ctx->speed_ring_from = s;
        if (dts)
            dts[k] = dtf;
        ctx->last_dt = dtf;
        t += dt;
        ++k;
        if (n_substeps)
            *n_substeps = k;
    }
    return MPM_OK;
}

mpm_status mpm_sync(mpm_ctx* ctx)
{
    if (!ctx)
        return MPM_EINVAL;
    return device_error(ctx);
}

mpm_status mpm_rebuild(mpm_ctx* ctx)
{
    if (!ctx)
        return MPM_EINVAL;
    mpm_status st = rebuild(ctx);
    if (st != MPM_OK)
        return st;
    return device_error(ctx);
}

mpm_status mpm_read_state(mpm_ctx* ctx, float* x, float* v, float* C, float* F, float* Jp, int on_device)
{
    TraceRange trace("mpm_read_state");
    if (!ctx)
        return MPM_EINVAL;
    float* outs[5] = {x, v, C, F, Jp};
    static const int W[5] = {3, 3, 9, 9, 1};
    int64_t n = ctx->n;
    for (int f = 0; f < 5 && n > 0; ++f) {
        if (!outs[f])
            continue;
        size_t bytes = (size_t)n * W[f] * 4;
        if (on_device) {
            launch_gather_out(ctx->pv[ctx->cur], n, f, outs[f], ctx->stream);
        } else {
            mpm_status st = ensure_stage(ctx, bytes);
            if (st != MPM_OK)
                return st;
            launch_gather_out(ctx->pv[ctx->cur], n, f, (float*)ctx->stage, ctx->stream);
            CK(cudaMemcpyAsync(outs[f], ctx->stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        }
        ctx->launches += 1;
    }
    CK(cudaGetLastError());
    return device_error(ctx);
}

mpm_status mpm_write_state(mpm_ctx* ctx, const float* x, const float* v, const float* C, const float* F,
                           const float* Jp, int on_device)
{
    if (!ctx)
        return MPM_EINVAL;
    if (v)
        forget_speeds(ctx);
    const float* ins[5] = {x, v, C, F, Jp};
    static const int W[5] = {3, 3, 9, 9, 1};
    int64_t n = ctx->n;
    for (int f = 0; f < 5 && n > 0; ++f) {
        if (!ins[f])
            continue;
        size_t bytes = (size_t)n * W[f] * 4;
        if (on_device) {
            launch_scatter_in(ctx->pv[ctx->cur], n, f, ins[f], ctx->stream);
        } else {
            mpm_status st = ensure_stage(ctx, bytes);
            if (st != MPM_OK)
                return st;
            CK(cudaMemcpyAsync(ctx->stage, ins[f], bytes, cudaMemcpyHostToDevice, ctx->stream));
            launch_scatter_in(ctx->pv[ctx->cur], n, f, (const float*)ctx->stage, ctx->stream);
            // the stage buffer is reused by the next field: order the copies
            CK(cudaStreamSynchronize(ctx->stream));
        }
        ctx->launches += 1;
    }
    if (F || Jp || !ctx->tau_valid) {
        launch_prepare_stress(ctx->sp, ctx->pv[ctx->cur], n, ctx->stream);
        ctx->launches += 1;
        ctx->tau_valid = true;
    }
    ctx->primed = false;
    if (x) {
        ctx->need_rebuild = true;
        ctx->keys_valid = false;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return MPM_OK;
}

int64_t mpm_num_particles(const mpm_ctx* ctx) { return ctx ? ctx->n : 0; }

const char* mpm_last_error(const mpm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mpm_status mpm_get_stats(const mpm_ctx* ctx, mpm_stats* out)
{
    if (!ctx || !out)
        return MPM_EINVAL;
    out->substeps = ctx->step;
    out->rebuilds = ctx->rebuilds;
    out->n_pblocks = ctx->n_pblocks;
    out->grid_capacity = ctx->grid_cap;
    out->particle_capacity = ctx->cap;
    out->kernel_launches = ctx->launches;
    return MPM_OK;
}

mpm_status mpm_read_order(mpm_ctx* ctx, uint32_t* keys, int32_t* ids, int on_device)
{
    if (!ctx)
        return MPM_EINVAL;
    if (ctx->cfg.no_sort)
        return fail(ctx, MPM_EINVAL, "mpm_read_order: the context does not sort (no_sort = 1)");
    if (!ctx->keys_valid)
        return fail(ctx, MPM_EINVAL, "mpm_read_order: no rebuild since the particles last changed");
    size_t bytes = (size_t)ctx->n * 4;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (keys && bytes)
        CK(cudaMemcpyAsync(keys, ctx->skeys, bytes, k, ctx->stream));
    if (ids && bytes)
        CK(cudaMemcpyAsync(ids, ctx->pv[ctx->cur].id, bytes, k, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MPM_OK;
}

mpm_status mpm_read_blocks(mpm_ctx* ctx, int32_t* slots, int64_t cap, int64_t* count)
{
    if (!ctx || !count || cap < 0)
        return MPM_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    *count = ctx->n_pblocks;
    int64_t m = cap < ctx->n_pblocks ? cap : ctx->n_pblocks;
    if (slots && m > 0)
        CK(cudaMemcpy(slots, ctx->pslot, (size_t)m * 4, cudaMemcpyDeviceToHost));
    return MPM_OK;
}

mpm_status mpm_debug_p2g(mpm_ctx* ctx, float dt, float* grid_out, int on_device)
{
    if (!ctx || !grid_out)
        return MPM_EINVAL;
    if (ctx->need_rebuild || ctx->n == 0) {
        mpm_status st = rebuild(ctx);
        if (st != MPM_OK)
            return st;
    }
    cudaStream_t s = ctx->stream;
    int64_t nodes = (int64_t)ctx->sp.res[0] * ctx->sp.res[1] * ctx->sp.res[2];
    size_t bytes = (size_t)nodes * 16;
    float* dense = grid_out;
    if (!on_device) {
        mpm_status st = ensure_stage(ctx, bytes);
        if (st != MPM_OK)
            return st;
        dense = (float*)ctx->stage;
    }
    CK(cudaMemsetAsync(dense, 0, bytes, s));
    if (!ctx->tau_valid) {
        launch_prepare_stress(ctx->sp, ctx->pv[ctx->cur], ctx->n, s);
        ctx->launches += 1;
        ctx->tau_valid = true;
    }
    if (ctx->primed && ctx->n_pblocks > 0) {   // fused mode keeps momentum there; rebuild it later
        CK(cudaMemsetAsync(ctx->grid[ctx->gcur], 0, (size_t)ctx->n_pblocks * 1024, s));
        ctx->primed = false;
    }
    GridView gv = grid_view(ctx);
    launch_p2g(ctx->sp, ctx->pv[ctx->cur], gv, ctx->n, dt, ctx->dstat, ctx->cfg.p2g_variant, s);
    launch_grid_to_dense(ctx->sp, gv.cur, ctx->pslot, ctx->n_pblocks, dense, s);
    ctx->launches += 2;
    if (ctx->n_pblocks > 0)
        CK(cudaMemsetAsync(gv.cur, 0, (size_t)ctx->n_pblocks * 1024, s));
    if (!on_device)
        CK(cudaMemcpyAsync(grid_out, dense, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaGetLastError());
    return device_error(ctx);
}

mpm_status mpm_set_p2g_variant(mpm_ctx* ctx, int variant)
{
    if (!ctx || variant < 0 || variant >= kP2GVariants)
        return MPM_EINVAL;
    if (ctx->aosoa && variant != P2G_CHUNK4 && variant != P2G_CHUNK8 && variant != P2G_NODE &&
        variant != P2G_CHUNK8S)
        return fail(ctx, MPM_EINVAL, "mpm_set_p2g_variant: the AoSoA layout has P2G variants 3, 4, 14 and 15 only");
    ctx->cfg.p2g_variant = variant;
    drop_graphs(ctx);
    return MPM_OK;
}

mpm_status mpm_set_layout(mpm_ctx* ctx, int aosoa)
{
    if (!ctx || (aosoa != 0 && aosoa != 1))
        return MPM_EINVAL;
    if (aosoa == ctx->aosoa)
        return MPM_OK;
    if (aosoa && ((ctx->cfg.p2g_variant != P2G_CHUNK4 && ctx->cfg.p2g_variant != P2G_CHUNK8 &&
                   ctx->cfg.p2g_variant != P2G_NODE && ctx->cfg.p2g_variant != P2G_CHUNK8S) ||
                  (ctx->cfg.g2p_variant != G2P_OCC && ctx->cfg.g2p_variant != G2P_OCCSW &&
                   ctx->cfg.g2p_variant != G2P_OCC10) || ctx->cfg.use_g2p2g ||
                  ctx->cfg.transfer != MPM_APIC ||
                  ctx->sp.cta_warps == 8))
        return fail(ctx, MPM_EINVAL,
                    "mpm_set_layout: AoSoA needs P2G variant 3, 4, 14 or 15, G2P variant 4, 6 or 7, separate APIC transfers and "
                    "2 or 4 warps per CTA");
    // convert the current particles into the other buffer, then make it current
    PartView dst = ctx->pv[1 - ctx->cur];
    dst.aosoa = aosoa;
    if (ctx->n > 0) {
        launch_relayout(ctx->pv[ctx->cur], dst, ctx->n, ctx->stream);
        ctx->launches += 1;
    }
    ctx->aosoa = aosoa;
    ctx->pv[0].aosoa = aosoa;
    ctx->pv[1].aosoa = aosoa;
    ctx->cur = 1 - ctx->cur;
    drop_graphs(ctx);
    CK(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_set_cta_warps(mpm_ctx* ctx, int warps)
{
    if (!ctx || (warps != 2 && warps != 4 && warps != 8))
        return MPM_EINVAL;
    if (ctx->aosoa && warps == 8)
        return fail(ctx, MPM_EINVAL, "mpm_set_cta_warps: the AoSoA layout runs 2 or 4 warps per CTA only");
    ctx->sp.cta_warps = warps;
    drop_graphs(ctx);
    return MPM_OK;
}

mpm_status mpm_set_resort_interval(mpm_ctx* ctx, int interval)
{
    if (!ctx || interval < 0)
        return MPM_EINVAL;
    ctx->cfg.resort_interval = interval;   // read on the host before each substep; no graph holds it
    return MPM_OK;
}

mpm_status mpm_set_g2p2g(mpm_ctx* ctx, int on)
{
    if (!ctx || (on != 0 && on != 1))
        return MPM_EINVAL;
    if (on && ctx->cfg.transfer == MPM_ASFLIP)
        return fail(ctx, MPM_EINVAL, "mpm_set_g2p2g: the fused transfer has no ASFLIP form");
    if (on && ctx->aosoa)
        return fail(ctx, MPM_EINVAL, "mpm_set_g2p2g: the fused transfer has no AoSoA form");
    if (ctx->cfg.use_g2p2g && !on && ctx->primed) {
        // back to separate phases: the next P2G needs a zero grid and the stress
        if (ctx->n_pblocks > 0)
            CK(cudaMemsetAsync(ctx->grid[ctx->gcur], 0, (size_t)ctx->n_pblocks * 1024, ctx->stream));
        ctx->primed = false;
    }
    if (!on && !ctx->tau_valid) {
        launch_prepare_stress(ctx->sp, ctx->pv[ctx->cur], ctx->n, ctx->stream);
        ctx->launches += 1;
        ctx->tau_valid = true;
    }
    ctx->cfg.use_g2p2g = on;
    return MPM_OK;
}

mpm_status mpm_set_g2p_variant(mpm_ctx* ctx, int variant)
{
    if (!ctx || variant < 0 || variant >= kG2PVariants)
        return MPM_EINVAL;
    if (ctx->aosoa && variant != G2P_OCC && variant != G2P_OCCSW && variant != G2P_OCC10)
        return fail(ctx, MPM_EINVAL, "mpm_set_g2p_variant: the AoSoA layout has G2P variants 4, 6 and 7 only");
    ctx->cfg.g2p_variant = variant;
    drop_graphs(ctx);
    return MPM_OK;
}

mpm_status mpm_profile_enable(mpm_ctx* ctx, int on)
{
    if (!ctx)
        return MPM_EINVAL;
    ctx->prof = on != 0;
    return MPM_OK;
}

mpm_status mpm_profile_read(mpm_ctx* ctx, double* ms, int64_t* launches, int n_phases)
{
    if (!ctx || n_phases < 0 || n_phases > MPM_PHASES)
        return MPM_EINVAL;
    prof_drain(ctx, 0);
    for (int i = 0; i < n_phases; ++i) {
        if (ms)
            ms[i] = ctx->prof_ms[i];
        if (launches)
            launches[i] = ctx->prof_launch[i];
    }
    for (int i = 0; i < MPM_PHASES; ++i) {
        ctx->prof_ms[i] = 0;
        ctx->prof_launch[i] = 0;
    }
    return MPM_OK;
}

mpm_status mpm_debug_svd(const float* F, float* U, float* sig, float* V, int64_t n)
{
    if (!F || n < 0)
        return MPM_EINVAL;
    launch_debug_svd(F, U, sig, V, n, 0);
    return cudaDeviceSynchronize() == cudaSuccess && cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

mpm_status mpm_debug_stress(const mpm_material* mat, const float* F, const float* Jp, float* tau, int64_t n)
{
    if (!mat || !F || !tau || n < 0 || !valid_material(*mat))
        return MPM_EINVAL;
    launch_debug_stress(make_mat_params(*mat), F, Jp, tau, n, 0);
    return cudaDeviceSynchronize() == cudaSuccess && cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

mpm_status mpm_debug_plasticity(const mpm_material* mat, float* F, float* Jp, int64_t n)
{
    if (!mat || !F || n < 0 || !valid_material(*mat))
        return MPM_EINVAL;
    launch_debug_plasticity(make_mat_params(*mat), F, Jp, n, 0);
    return cudaDeviceSynchronize() == cudaSuccess && cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

mpm_status mpm_debug_red_rate(void* grid, int64_t nodes, int64_t threads, int32_t reds_per_thread, int32_t pattern,
                              void* stream)
{
    if (!grid || nodes < 32 || nodes % 32 != 0 || threads < 32 || threads % 32 != 0 || threads > (int64_t)1 << 31 ||
        reds_per_thread < 1 || reds_per_thread > 4096 || pattern < 0 || pattern > 3 ||
        ((uintptr_t)grid & 15u) != 0)
        return MPM_EINVAL;
    return launch_debug_red_rate(static_cast<float4*>(grid), nodes, threads, reds_per_thread, pattern,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? MPM_OK
               : MPM_ECUDA;
}

mpm_status mpm_debug_wait_timeout(int max_iter)
{
    if (max_iter < 1 || max_iter > (1 << 16))
        return MPM_EINVAL;
    uint32_t* err = nullptr;
    if (cudaMalloc(&err, 4) != cudaSuccess)
        return MPM_ENOMEM;
    uint32_t h = 0;
    cudaMemset(err, 0, 4);
    launch_debug_wait_timeout(max_iter, err, 0);
    cudaError_t e = cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return MPM_ECUDA;
    return (h & ST_TIMEOUT) ? MPM_ETIMEOUT : MPM_OK;
}

}  // extern "C"
