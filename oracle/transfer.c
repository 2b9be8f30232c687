/*
 * Oracle (test infrastructure only): the three essential phases of one
 * explicit MLS-MPM substep (Sec. 4: transfer-particle-to-grid, update-grid,
 * transfer-grid-to-particle), on a plain dense box of grid nodes in FP64.
 *
 * No sorting, blocking, hashing, free zone or warp reduction: those change
 * only speed and summation order (Sec. 4.2), so the oracle leaves them out.
 *
 * Formulas (MLS-MPM, Hu et al. 2018, named in Sec. 6), with h = dx:
 *   P2G   m_i += w_ip m_p
 *         p_i += w_ip [ m_p v_p + (m_p C_p - (4 dt V_p / h^2) tau_p)(x_i - x_p) ]
 *   grid  v_i = p_i / m_i + dt g  if m_i > 0, else 0; then the walls:
 *         sticky: v_i = 0 on wall nodes; slip: the velocity component that
 *         points into a wall is zeroed, axis by axis.  A node is a wall node
 *         on axis a if i_a < wall or i_a >= res_a - wall.
 *   G2P   v_p = sum w_ip v_i,  C_p = (4 / h^2) sum w_ip v_i (x_i - x_p)^T,
 *         x_p += dt v_p,  F_p <- (I + dt C_p) F_p, then the return map;
 *         fluid: J_p <- (1 + dt tr C_p) J_p and F is left unchanged.
 * m_p = rho_mat * V_p.
 *
 * ASFLIP (Fei et al. 2021; the integrator of the paper's fountain, Sec. 6.5)
 * changes only the particle velocity and position of G2P.  With
 * vbar_p = sum w_ip v_i (the new grid velocity, as above) and
 * v0_p = sum w_ip v0_i, v0_i = p_i / m_i the grid velocity before any force:
 *         v_p <- vbar_p + alpha (v_p - v0_p)
 *         x_p <- x_p + dt [ vbar_p + beta alpha (v_p(old) - v0_p) ]
 * with beta = beta_min if the particle is compressed and beta_max otherwise.
 * Compressed means J < 1 - 1e-4 (J = det F, the tracked J for the fluid,
 * taken before this G2P): the sand return map sets every particle under
 * tension to J = 1 exactly, where the rounding of det F (FP32 ~1e-6) would
 * otherwise choose beta at random; such particles count as not compressed.
 * C_p, F_p and J_p are updated exactly as in APIC.  alpha = beta = 0 is APIC.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define AT(M, r, c) (M)[3 * (r) + (c)]

static double det3(const double* M)
{
    return AT(M, 0, 0) * (AT(M, 1, 1) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 1)) -
           AT(M, 0, 1) * (AT(M, 1, 0) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 0)) +
           AT(M, 0, 2) * (AT(M, 1, 0) * AT(M, 2, 1) - AT(M, 1, 1) * AT(M, 2, 0));
}

static void base_and_weights(const double* xp, double inv_dx, int32_t base[3],
                             double fx[3], double w[3][3])
{
    for (int a = 0; a < 3; ++a) {
        double X = xp[a] * inv_dx;
        double b = floor(X - 0.5);
        base[a] = (int32_t)b;
        fx[a] = X - b;
        orc_bspline_weights(fx[a], w[a]);
    }
}

int orc_grid_bounds(int64_t n, const double* x, double dx, int32_t lo[3], int32_t dim[3])
{
    double inv_dx = 1.0 / dx;
    int32_t mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
    for (int64_t p = 0; p < n; ++p)
        for (int a = 0; a < 3; ++a) {
            int32_t b = (int32_t)floor(x[3 * p + a] * inv_dx - 0.5);
            if (p == 0 || b < mn[a]) mn[a] = b;
            if (p == 0 || b + 2 > mx[a]) mx[a] = b + 2;
        }
    for (int a = 0; a < 3; ++a) {
        lo[a] = mn[a];
        dim[a] = n > 0 ? mx[a] - mn[a] + 1 : 0;
    }
    return ORC_OK;
}

static int in_domain(const orc_config* cfg, const int32_t base[3])
{
    for (int a = 0; a < 3; ++a)
        if (base[a] < 0 || base[a] + 2 >= cfg->res[a])
            return 0;
    return 1;
}

int orc_p2g(const orc_config* cfg, const orc_material* mats, int64_t n,
            const double* x, const double* v, const double* C, const double* F,
            const double* Jp, const double* vol, const int32_t* mat, double dt,
            orc_grid* g)
{
    double h = cfg->dx, inv_dx = 1.0 / h;
    int status = ORC_OK;
    for (int64_t p = 0; p < n; ++p) {
        const orc_material* M = &mats[mat[p]];
        int32_t base[3];
        double f[3], w[3][3], tau[9], A[9];
        base_and_weights(&x[3 * p], inv_dx, base, f, w);
        if (!in_domain(cfg, base)) {
            status = ORC_EDOMAIN;
            continue;
        }
        double mp = M->rho * vol[p];
        orc_kirchhoff(M, &F[9 * p], Jp[p], tau);
        double k = 4.0 * dt * vol[p] / (h * h);
        for (int e = 0; e < 9; ++e)
            A[e] = mp * C[9 * p + e] - k * tau[e];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double d[3] = {(i - f[0]) * h, (j - f[1]) * h, (l - f[2]) * h};
                    int32_t gi = base[0] + i - g->lo[0];
                    int32_t gj = base[1] + j - g->lo[1];
                    int32_t gl = base[2] + l - g->lo[2];
                    if (gi < 0 || gj < 0 || gl < 0 || gi >= g->dim[0] || gj >= g->dim[1] || gl >= g->dim[2]) {
                        status = ORC_EDOMAIN;
                        continue;
                    }
                    int64_t id = gi + (int64_t)g->dim[0] * (gj + (int64_t)g->dim[1] * gl);
                    g->m[id] += wt * mp;
                    for (int a = 0; a < 3; ++a) {
                        double Ad = AT(A, a, 0) * d[0] + AT(A, a, 1) * d[1] + AT(A, a, 2) * d[2];
                        g->p[3 * id + a] += wt * (mp * v[3 * p + a] + Ad);
                    }
                }
    }
    return status;
}

void orc_grid_update(const orc_config* cfg, double dt, orc_grid* g)
{
    int64_t nn = (int64_t)g->dim[0] * g->dim[1] * g->dim[2];
    for (int64_t id = 0; id < nn; ++id) {
        int32_t c[3];
        c[0] = (int32_t)(id % g->dim[0]) + g->lo[0];
        c[1] = (int32_t)((id / g->dim[0]) % g->dim[1]) + g->lo[1];
        c[2] = (int32_t)(id / ((int64_t)g->dim[0] * g->dim[1])) + g->lo[2];
        double* vi = &g->p[3 * id];
        if (!(g->m[id] > 0.0)) {
            vi[0] = vi[1] = vi[2] = 0.0;
            if (g->v0)
                g->v0[3 * id] = g->v0[3 * id + 1] = g->v0[3 * id + 2] = 0.0;
            continue;
        }
        if (g->v0)
            for (int a = 0; a < 3; ++a)
                g->v0[3 * id + a] = vi[a] / g->m[id];
        for (int a = 0; a < 3; ++a)
            vi[a] = vi[a] / g->m[id] + dt * cfg->gravity[a];
        for (int a = 0; a < 3; ++a) {
            int low = c[a] < cfg->wall, high = c[a] >= cfg->res[a] - cfg->wall;
            if (cfg->boundary == ORC_STICKY) {
                if (low || high) {
                    vi[0] = vi[1] = vi[2] = 0.0;
                    break;
                }
            } else {
                if (low && vi[a] < 0.0) vi[a] = 0.0;
                if (high && vi[a] > 0.0) vi[a] = 0.0;
            }
        }
    }
}

int orc_g2p(const orc_config* cfg, const orc_material* mats, int64_t n,
            double* x, double* v, double* C, double* F, double* Jp,
            const int32_t* mat, double dt, const orc_grid* g)
{
    double h = cfg->dx, inv_dx = 1.0 / h;
    int status = ORC_OK;
    int asflip = cfg->transfer == ORC_ASFLIP;
    if (asflip && !g->v0)
        return ORC_EINVAL;
    for (int64_t p = 0; p < n; ++p) {
        const orc_material* M = &mats[mat[p]];
        int32_t base[3];
        double f[3], w[3][3], vp[3] = {0, 0, 0}, B[9] = {0}, v0p[3] = {0, 0, 0};
        base_and_weights(&x[3 * p], inv_dx, base, f, w);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double d[3] = {(i - f[0]) * h, (j - f[1]) * h, (l - f[2]) * h};
                    int32_t gi = base[0] + i - g->lo[0];
                    int32_t gj = base[1] + j - g->lo[1];
                    int32_t gl = base[2] + l - g->lo[2];
                    if (gi < 0 || gj < 0 || gl < 0 || gi >= g->dim[0] || gj >= g->dim[1] || gl >= g->dim[2]) {
                        status = ORC_EDOMAIN;
                        continue;
                    }
                    int64_t id = gi + (int64_t)g->dim[0] * (gj + (int64_t)g->dim[1] * gl);
                    const double* vi = &g->p[3 * id];
                    for (int a = 0; a < 3; ++a) {
                        vp[a] += wt * vi[a];
                        for (int b = 0; b < 3; ++b)
                            AT(B, a, b) += wt * vi[a] * d[b];
                        if (asflip)
                            v0p[a] += wt * g->v0[3 * id + a];
                    }
                }
        double* Cp = &C[9 * p];
        for (int e = 0; e < 9; ++e)
            Cp[e] = 4.0 * inv_dx * inv_dx * B[e];
        if (asflip) {
            double J = M->kind == ORC_FLUID ? Jp[p] : det3(&F[9 * p]);
            double beta = J < 1.0 - cfg->flip_compress_margin ? cfg->flip_beta_min : cfg->flip_beta_max;
            for (int a = 0; a < 3; ++a) {
                double dv = v[3 * p + a] - v0p[a];
                x[3 * p + a] += dt * (vp[a] + beta * cfg->flip_alpha * dv);
                v[3 * p + a] = vp[a] + cfg->flip_alpha * dv;
            }
        } else {
            for (int a = 0; a < 3; ++a) {
                v[3 * p + a] = vp[a];
                x[3 * p + a] += dt * vp[a];
            }
        }
        if (M->kind == ORC_FLUID) {
            Jp[p] *= 1.0 + dt * (AT(Cp, 0, 0) + AT(Cp, 1, 1) + AT(Cp, 2, 2));
            continue;
        }
        double* Fp = &F[9 * p];
        double Fn[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int k = 0; k < 3; ++k)
                    s += ((a == k ? 1.0 : 0.0) + dt * AT(Cp, a, k)) * AT(Fp, k, b);
                AT(Fn, a, b) = s;
            }
        memcpy(Fp, Fn, sizeof(Fn));
        orc_plasticity(M, Fp, &Jp[p]);
    }
    return status;
}

int orc_substep(const orc_config* cfg, const orc_material* mats, int64_t n,
                double* x, double* v, double* C, double* F, double* Jp,
                const double* vol, const int32_t* mat, double dt)
{
    orc_grid g;
    orc_grid_bounds(n, x, cfg->dx, g.lo, g.dim);
    int64_t nn = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
    g.m = (double*)calloc(nn > 0 ? nn : 1, sizeof(double));
    g.p = (double*)calloc(nn > 0 ? 3 * nn : 1, sizeof(double));
    g.v0 = cfg->transfer == ORC_ASFLIP ? (double*)calloc(nn > 0 ? 3 * nn : 1, sizeof(double)) : NULL;
    if (!g.m || !g.p || (cfg->transfer == ORC_ASFLIP && !g.v0)) {
        free(g.m);
        free(g.p);
        free(g.v0);
        return ORC_EINVAL;
    }
    int s1 = orc_p2g(cfg, mats, n, x, v, C, F, Jp, vol, mat, dt, &g);
    orc_grid_update(cfg, dt, &g);
    int s2 = orc_g2p(cfg, mats, n, x, v, C, F, Jp, mat, dt, &g);
    free(g.m);
    free(g.p);
    free(g.v0);
    return s1 != ORC_OK ? s1 : s2;
}

void orc_p2g_node(const orc_config* cfg, const orc_material* mats, int64_t n,
                  const double* x, const double* v, const double* C, const double* F,
                  const double* Jp, const double* vol, const int32_t* mat, double dt,
                  const int32_t node[3], double out[4])
{
    double h = cfg->dx, inv_dx = 1.0 / h;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        int32_t base[3];
        double f[3], w[3][3], tau[9];
        base_and_weights(&x[3 * p], inv_dx, base, f, w);
        int32_t o[3];
        int hit = 1;
        for (int a = 0; a < 3; ++a) {
            o[a] = node[a] - base[a];
            if (o[a] < 0 || o[a] > 2)
                hit = 0;
        }
        if (!hit)
            continue;
        const orc_material* M = &mats[mat[p]];
        double mp = M->rho * vol[p];
        orc_kirchhoff(M, &F[9 * p], Jp[p], tau);
        double k = 4.0 * dt * vol[p] / (h * h);
        double wt = w[0][o[0]] * w[1][o[1]] * w[2][o[2]];
        double d[3] = {(o[0] - f[0]) * h, (o[1] - f[1]) * h, (o[2] - f[2]) * h};
        out[0] += wt * mp;
        for (int a = 0; a < 3; ++a) {
            double Ad = 0;
            for (int b = 0; b < 3; ++b)
                Ad += (mp * C[9 * p + 3 * a + b] - k * tau[3 * a + b]) * d[b];
            out[1 + a] += wt * (mp * v[3 * p + a] + Ad);
        }
    }
}
