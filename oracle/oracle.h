/*
 * FP64 CPU oracle for one explicit MLS-MPM substep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  The
 * product library never links it and shares no header, helper, table or
 * constant with it.
 *
 * What it computes (paper: "Principles towards Real-Time Simulation of
 * Material Point Method on Modern GPUs", Sec. 4 and Sec. 6): the five-phase
 * explicit MLS-MPM time step (Sec. 4, phase list) with quadratic B-spline
 * weights (Sec. 3.1), the particle code of Sec. 4 (block code in the high
 * bits, cell code in the low bits), the histogram sort key (the block's
 * index, then the cell code; Sec. 4.2.2), and the physical-block set
 * (gblocks plus their 3x3x3 neighbours, Sec. 4 and Sec. 4.2.1).  The paper
 * names MLS-MPM [Hu et al. 2018] but prints no equation, so the transfer and
 * constitutive formulas are the cited literature's, written out plainly:
 *   - MLS-MPM transfers (Hu et al. 2018): D^-1 = 4/dx^2.
 *   - fixed-corotated elasticity (Stomakhin et al. 2012).
 *   - snow: fixed-corotated on F_E with exp(xi (1 - Jp)) hardening and
 *     singular-value clamping (Stomakhin et al. 2013).
 *   - weakly compressible fluid: p = K (J^-gamma - 1) (Tampubolon et al. 2017).
 *   - Drucker-Prager sand: Hencky-strain St. Venant-Kirchhoff stress and
 *     the three-case return map (Klar et al. 2016).
 * Where the paper leaves a point open, the reading taken is stated at the
 * function that implements it.
 *
 * Layout: particle arrays are AoS row-major doubles: x[n*3], v[n*3],
 * C[n*9] (C[p*9 + 3*a + b] = C_ab), F[n*9], Jp[n].  Grid arrays are a dense
 * box of nodes with global origin lo[3] and extent dim[3]; node (i,j,k) of
 * the box is global node lo + (i,j,k) and sits at linear index
 * i + dim0*(j + dim1*k).
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ELASTIC = 0, ORC_FLUID = 1, ORC_SNOW = 2, ORC_SAND = 3, ORC_NACC = 4, ORC_NHSAND = 5 };
enum { ORC_STICKY = 0, ORC_SLIP = 1 };
enum { ORC_OK = 0, ORC_EDOMAIN = 4, ORC_EINVAL = 1 };

typedef struct {
    int32_t kind;
    double E;          /* Young's modulus; for ORC_FLUID the bulk modulus K */
    double nu;         /* Poisson ratio (unused by ORC_FLUID) */
    double rho;        /* density */
    double gamma;      /* fluid exponent */
    double theta_c;    /* snow critical compression */
    double theta_s;    /* snow critical stretch */
    double hardening;  /* snow hardening coefficient xi */
    double friction_deg; /* sand friction angle phi in degrees */
    double friction_M; /* NACC: slope M of the critical state line */
    double cohesion;   /* NACC: cohesion beta */
    double alpha0;     /* NACC: initial hardening state alpha (ln of the plastic volume ratio) */
} orc_material;

enum { ORC_APIC = 0, ORC_ASFLIP = 1 };

typedef struct {
    int32_t res[3];    /* grid nodes per axis */
    double dx;
    int32_t boundary;  /* ORC_STICKY or ORC_SLIP */
    int32_t wall;      /* wall layer thickness in nodes */
    double gravity[3];
    int32_t transfer;  /* ORC_APIC, or ORC_ASFLIP (the integrator of the paper's
                          fountain, Sec. 6.5, after Fei et al. 2021) */
    double flip_alpha; /* ASFLIP: weight of the particle's own velocity change */
    double flip_beta_min, flip_beta_max; /* ASFLIP: positional weight when the particle
                          is compressed (J < 1 - flip_compress_margin) / not compressed */
    double flip_compress_margin; /* ASFLIP: m >= 0 in the compressed-state test J < 1 - m
                          (0 is the plain test J < 1) */
} orc_config;

typedef struct {
    int32_t lo[3];
    int32_t dim[3];
    double* m;         /* dim0*dim1*dim2 masses */
    double* p;         /* 3 per node: momentum after P2G, velocity after update */
    double* v0;        /* NULL, or 3 per node: the update writes p/m before any force */
} orc_grid;

/* Quadratic B-spline weights for fractional offset f in [0.5, 1.5). */
void orc_bspline_weights(double f, double w[3]);

/* Rotation-variant SVD F = U diag(sig) V^T, det U = det V = +1,
 * sig[0] >= sig[1] >= |sig[2]|, sig[2] carries the sign of det F. */
void orc_svd3(const double F[9], double U[9], double sig[3], double V[9]);

/* Lame parameters from (E, nu). */
void orc_lame(double E, double nu, double* mu, double* la);

/* Dilatational (p-wave) speed of a material at rest. */
double orc_wave_speed(const orc_material* mat);

/* Adaptive step size: min(dt_max, cfl dx / (v_bound + max wave speed of
 * mats[0..n_mats-1])). */
double orc_cfl_dt(const orc_config* cfg, const orc_material* mats, int n_mats, double v_bound, double cfl,
                  double dt_max);

/* Kirchhoff stress tau = P F^T of one particle.  Jp is the snow (and NACC)
 * plastic volume ratio, or the fluid J; ignored for elastic and sand.
 * ORC_NACC: E is the bulk modulus kappa, hardening is xi. */
void orc_kirchhoff(const orc_material* mat, const double F[9], double Jp, double tau[9]);

/* Return mapping applied to the trial F at the end of G2P (snow clamp,
 * Drucker-Prager projection; identity for elastic).  Fluid is handled by
 * the J update in orc_g2p. */
void orc_plasticity(const orc_material* mat, double F[9], double* Jp);

/* Smallest dense box covering every particle's 3x3x3 stencil. */
int orc_grid_bounds(int64_t n, const double* x, double dx, int32_t lo[3], int32_t dim[3]);

/* Phase 3, particle-to-grid: adds mass and MLS momentum (with the stress
 * impulse) into g, which the caller has zeroed. */
int orc_p2g(const orc_config* cfg, const orc_material* mats, int64_t n,
            const double* x, const double* v, const double* C, const double* F,
            const double* Jp, const double* vol, const int32_t* mat, double dt,
            orc_grid* g);

/* Phase 4, grid update: p -> v = p/m + dt g for m > 0, else 0, then the
 * wall boundary condition.  In place on g->p. */
void orc_grid_update(const orc_config* cfg, double dt, orc_grid* g);

/* Phase 5, grid-to-particle with the F update and the return mapping.
 * ASFLIP (cfg->transfer) needs g->v0 filled by orc_grid_update. */
int orc_g2p(const orc_config* cfg, const orc_material* mats, int64_t n,
            double* x, double* v, double* C, double* F, double* Jp,
            const int32_t* mat, double dt, const orc_grid* g);

/* One substep: bounds, P2G, grid update, G2P.  Allocates its own grid. */
int orc_substep(const orc_config* cfg, const orc_material* mats, int64_t n,
                double* x, double* v, double* C, double* F, double* Jp,
                const double* vol, const int32_t* mat, double dt);

/* Grid mass and momentum of one global node after P2G, summed particle by
 * particle over all n (for sampled checks at sizes where a full grid is
 * not wanted).  out[0] = m, out[1..3] = momentum. */
void orc_p2g_node(const orc_config* cfg, const orc_material* mats, int64_t n,
                  const double* x, const double* v, const double* C, const double* F,
                  const double* Jp, const double* vol, const int32_t* mat, double dt,
                  const int32_t node[3], double out[4]);

/* Particle code / sort key of Sec. 4 and Sec. 4.2.2, computed from FP32
 * positions in FP32 arithmetic (the precision the GPU path decides in):
 * base = floor(x * inv_dx - 0.5) per axis, block = base >> 2,
 * cell = base & 3, key = (morton(block, L bits per axis) << 6) | morton(cell).
 * Returns ORC_EDOMAIN if some base is negative or block >= 2^L. */
int orc_particle_keys(int64_t n, const float* x, float inv_dx, int32_t L, uint32_t* keys);

/* Stable ascending sort of keys, ties broken by original index.
 * perm[r] = original index of the r-th smallest. */
void orc_stable_sort(int64_t n, const uint32_t* keys, int32_t* perm);

/* Physical blocks (Sec. 4, Sec. 4.2.1): the Morton slots of every block in
 * the 3x3x3 neighbourhood of a block holding a particle, clipped to the
 * 2^L domain, in ascending order (so the index is the rank of the Morton
 * code).  Returns the count; out may be NULL to count only. */
int64_t orc_pblocks(int64_t n, const uint32_t* keys, int32_t L, int32_t* out);

/* Differentiable elastic substep (fixed-corotated, per-particle E, common
 * nu and rho).  State per particle: x[3] v[3] C[9] F[9] (24 doubles).
 * orc_diff_adjoint maps the adjoint of the output state to the adjoint of
 * the input state (written to g_in) and adds dL/dE into gE. */
int orc_diff_forward(const orc_config* cfg, double nu, double rho, int64_t n, const double* vol, const double* E,
                     double dt, const double* s_in, double* s_out);
int orc_diff_adjoint(const orc_config* cfg, double nu, double rho, int64_t n, const double* vol, const double* E,
                     double dt, const double* s_in, const double* g_out, double* g_in, double* gE);

#ifdef __cplusplus
}
#endif
#endif
