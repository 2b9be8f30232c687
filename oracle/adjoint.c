/*
 * Oracle (test infrastructure only): one differentiable elastic MLS-MPM
 * substep and its reverse-mode adjoint, in FP64.
 *
 * The paper does not differentiate the simulation; the differentiable rollout
 * is an addition on top of the same substep (Sec. 4 phases: P2G, grid update,
 * G2P).  Model: fixed-corotated elasticity with a per-particle Young's modulus
 * E_p and a common Poisson ratio nu and density rho (mu, lambda from E, nu).
 *
 * State of one particle: s = (x[3], v[3], C[9], F[9]), 24 doubles, row-major.
 * orc_diff_adjoint takes the adjoint sbar' of the state after the substep and
 * returns sbar of the state before it, and adds dL/dE_p into gE.
 *
 * The reverse pass follows the forward phases backwards (G2P, grid update,
 * P2G), by the chain rule, with one deliberate shortcut: the Jacobian of the
 * Kirchhoff stress tau(F) is taken by central differences in FP64 (step
 * 1e-6), which is plain and obviously consistent with orc_kirchhoff.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define AT(M, r, c) (M)[3 * (r) + (c)]

typedef struct {
    int32_t base[3];
    double f[3];
    double w[3][3];   /* w[a][i]: 1D weight of node offset i along axis a */
    double dw[3][3];  /* dW/df */
} stencil;

static void make_stencil(const double* x, double inv_dx, stencil* s)
{
    for (int a = 0; a < 3; ++a) {
        double X = x[a] * inv_dx;
        double b = floor(X - 0.5);
        s->base[a] = (int32_t)b;
        double f = X - b;
        s->f[a] = f;
        orc_bspline_weights(f, s->w[a]);
        s->dw[a][0] = -(1.5 - f);
        s->dw[a][1] = -2.0 * (f - 1.0);
        s->dw[a][2] = f - 0.5;
    }
}

static int64_t node_index(const orc_grid* g, const stencil* s, int i, int j, int k)
{
    int32_t gi = s->base[0] + i - g->lo[0], gj = s->base[1] + j - g->lo[1], gk = s->base[2] + k - g->lo[2];
    if (gi < 0 || gj < 0 || gk < 0 || gi >= g->dim[0] || gj >= g->dim[1] || gk >= g->dim[2])
        return -1;
    return gi + (int64_t)g->dim[0] * (gj + (int64_t)g->dim[1] * gk);
}

static orc_material elastic(double E, double nu, double rho)
{
    orc_material m;
    memset(&m, 0, sizeof(m));
    m.kind = ORC_ELASTIC;
    m.E = E;
    m.nu = nu;
    m.rho = rho;
    return m;
}

/* unpack a 24-double state into the AoS arrays the forward oracle uses */
static void unpack(int64_t n, const double* s, double* x, double* v, double* C, double* F)
{
    for (int64_t p = 0; p < n; ++p) {
        memcpy(&x[3 * p], &s[24 * p], 3 * sizeof(double));
        memcpy(&v[3 * p], &s[24 * p + 3], 3 * sizeof(double));
        memcpy(&C[9 * p], &s[24 * p + 6], 9 * sizeof(double));
        memcpy(&F[9 * p], &s[24 * p + 15], 9 * sizeof(double));
    }
}

static void pack(int64_t n, const double* x, const double* v, const double* C, const double* F, double* s)
{
    for (int64_t p = 0; p < n; ++p) {
        memcpy(&s[24 * p], &x[3 * p], 3 * sizeof(double));
        memcpy(&s[24 * p + 3], &v[3 * p], 3 * sizeof(double));
        memcpy(&s[24 * p + 6], &C[9 * p], 9 * sizeof(double));
        memcpy(&s[24 * p + 15], &F[9 * p], 9 * sizeof(double));
    }
}

/* forward substep with per-particle E (elastic); grid box sized from s_in */
int orc_diff_forward(const orc_config* cfg, double nu, double rho, int64_t n, const double* vol, const double* E,
                     double dt, const double* s_in, double* s_out)
{
    if (cfg->transfer != ORC_APIC)
        return ORC_EINVAL;   /* the reverse pass below is APIC's */
    double* x = malloc(sizeof(double) * 3 * n);
    double* v = malloc(sizeof(double) * 3 * n);
    double* C = malloc(sizeof(double) * 9 * n);
    double* F = malloc(sizeof(double) * 9 * n);
    double* Jp = malloc(sizeof(double) * n);
    int32_t* mat = malloc(sizeof(int32_t) * n);
    orc_material* mats = malloc(sizeof(orc_material) * n);
    unpack(n, s_in, x, v, C, F);
    for (int64_t p = 0; p < n; ++p) {
        Jp[p] = 1.0;
        mat[p] = (int32_t)p;
        mats[p] = elastic(E[p], nu, rho);
    }
    int st = orc_substep(cfg, mats, n, x, v, C, F, Jp, vol, mat, dt);
    pack(n, x, v, C, F, s_out);
    free(x); free(v); free(C); free(F); free(Jp); free(mat); free(mats);
    return st;
}

/* tau(F) for one particle, and its Jacobian contracted with taubar:
 * Fbar[ab] = sum_cd taubar[cd] d tau[cd] / d F[ab] (central differences) */
static void stress_vjp(const orc_material* m, const double F[9], const double taubar[9], double Fbar[9])
{
    const double h = 1e-6;
    for (int e = 0; e < 9; ++e) {
        double Fp[9], Fm[9], tp[9], tm[9];
        memcpy(Fp, F, sizeof(Fp));
        memcpy(Fm, F, sizeof(Fm));
        Fp[e] += h;
        Fm[e] -= h;
        orc_kirchhoff(m, Fp, 1.0, tp);
        orc_kirchhoff(m, Fm, 1.0, tm);
        double s = 0;
        for (int c = 0; c < 9; ++c)
            s += taubar[c] * (tp[c] - tm[c]) / (2.0 * h);
        Fbar[e] = s;
    }
}

int orc_diff_adjoint(const orc_config* cfg, double nu, double rho, int64_t n, const double* vol, const double* E,
                     double dt, const double* s_in, const double* g_out, double* g_in, double* gE)
{
    if (cfg->transfer != ORC_APIC)
        return ORC_EINVAL;
    const double h = cfg->dx, inv_dx = 1.0 / h, D = 4.0 * inv_dx * inv_dx;
    double* x = malloc(sizeof(double) * 3 * n);
    double* v = malloc(sizeof(double) * 3 * n);
    double* C = malloc(sizeof(double) * 9 * n);
    double* F = malloc(sizeof(double) * 9 * n);
    unpack(n, s_in, x, v, C, F);
    /* ---- forward recomputation of the grid ---- */
    orc_grid g;
    g.v0 = NULL;
    orc_grid_bounds(n, x, h, g.lo, g.dim);
    int64_t nn = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
    g.m = calloc(nn, sizeof(double));
    g.p = calloc(3 * nn, sizeof(double));
    orc_material* mats = malloc(sizeof(orc_material) * n);
    int32_t* mat = malloc(sizeof(int32_t) * n);
    double* Jp = malloc(sizeof(double) * n);
    for (int64_t p = 0; p < n; ++p) {
        mats[p] = elastic(E[p], nu, rho);
        mat[p] = (int32_t)p;
        Jp[p] = 1.0;
    }
    int st = orc_p2g(cfg, mats, n, x, v, C, F, Jp, vol, mat, dt, &g);
    double* P = malloc(sizeof(double) * 3 * nn);  /* momentum before the update */
    memcpy(P, g.p, sizeof(double) * 3 * nn);
    orc_grid_update(cfg, dt, &g);                   /* g.p now holds v_i */
    /* ---- reverse G2P ---- */
    double* vbar_i = calloc(3 * nn, sizeof(double));
    memset(g_in, 0, sizeof(double) * 24 * n);
    for (int64_t p = 0; p < n; ++p) {
        const double* xb1 = &g_out[24 * p];
        const double* vb1 = &g_out[24 * p + 3];
        const double* Cb1 = &g_out[24 * p + 6];
        const double* Fb1 = &g_out[24 * p + 15];
        stencil S;
        make_stencil(&x[3 * p], inv_dx, &S);
        /* recompute C' */
        double Cn[9] = {0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    int64_t id = node_index(&g, &S, i, j, k);
                    if (id < 0)
                        continue;
                    double wt = S.w[0][i] * S.w[1][j] * S.w[2][k];
                    double d[3] = {(i - S.f[0]) * h, (j - S.f[1]) * h, (k - S.f[2]) * h};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            AT(Cn, a, b) += D * wt * g.p[3 * id + a] * d[b];
                }
        const double* Fp = &F[9 * p];
        double* xb = &g_in[24 * p];
        double* Fb = &g_in[24 * p + 15];
        /* F' = (I + dt C') F */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int c = 0; c < 3; ++c)
                    s += ((c == a ? 1.0 : 0.0) + dt * AT(Cn, c, a)) * AT(Fb1, c, b);
                AT(Fb, a, b) = s;
            }
        double Ct[9];   /* total adjoint of C' */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int c = 0; c < 3; ++c)
                    s += AT(Fb1, a, c) * AT(Fp, b, c);
                AT(Ct, a, b) = AT(Cb1, a, b) + dt * s;
            }
        double vt[3];   /* total adjoint of v' (x' = x + dt v') */
        for (int a = 0; a < 3; ++a) {
            xb[a] = xb1[a];
            vt[a] = vb1[a] + dt * xb1[a];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    int64_t id = node_index(&g, &S, i, j, k);
                    if (id < 0)
                        continue;
                    double wt = S.w[0][i] * S.w[1][j] * S.w[2][k];
                    double gw[3] = {inv_dx * S.dw[0][i] * S.w[1][j] * S.w[2][k],
                                    inv_dx * S.w[0][i] * S.dw[1][j] * S.w[2][k],
                                    inv_dx * S.w[0][i] * S.w[1][j] * S.dw[2][k]};
                    double d[3] = {(i - S.f[0]) * h, (j - S.f[1]) * h, (k - S.f[2]) * h};
                    const double* vi = &g.p[3 * id];
                    double Cd[3], CtTv[3], vCd = 0, vtv = 0;
                    for (int a = 0; a < 3; ++a) {
                        Cd[a] = AT(Ct, a, 0) * d[0] + AT(Ct, a, 1) * d[1] + AT(Ct, a, 2) * d[2];
                        CtTv[a] = AT(Ct, 0, a) * vi[0] + AT(Ct, 1, a) * vi[1] + AT(Ct, 2, a) * vi[2];
                    }
                    for (int a = 0; a < 3; ++a) {
                        vbar_i[3 * id + a] += wt * (vt[a] + D * Cd[a]);
                        vtv += vt[a] * vi[a];
                        vCd += vi[a] * Cd[a];
                    }
                    for (int a = 0; a < 3; ++a)
                        xb[a] += gw[a] * (vtv + D * vCd) - D * wt * CtTv[a];
                }
    }
    /* ---- reverse grid update ---- */
    double* Pbar = calloc(3 * nn, sizeof(double));
    double* mbar = calloc(nn, sizeof(double));
    for (int64_t id = 0; id < nn; ++id) {
        if (!(g.m[id] > 0.0))
            continue;
        int32_t c[3];
        c[0] = (int32_t)(id % g.dim[0]) + g.lo[0];
        c[1] = (int32_t)((id / g.dim[0]) % g.dim[1]) + g.lo[1];
        c[2] = (int32_t)(id / ((int64_t)g.dim[0] * g.dim[1])) + g.lo[2];
        double keep[3] = {1, 1, 1};
        for (int a = 0; a < 3; ++a) {
            int low = c[a] < cfg->wall, high = c[a] >= cfg->res[a] - cfg->wall;
            double vfree = P[3 * id + a] / g.m[id] + dt * cfg->gravity[a];
            if (cfg->boundary == ORC_STICKY) {
                if (low || high)
                    keep[0] = keep[1] = keep[2] = 0;
            } else {
                if ((low && vfree < 0.0) || (high && vfree > 0.0))
                    keep[a] = 0;
            }
        }
        for (int a = 0; a < 3; ++a) {
            double vb = keep[a] * vbar_i[3 * id + a];
            Pbar[3 * id + a] = vb / g.m[id];
            mbar[id] -= vb * P[3 * id + a] / (g.m[id] * g.m[id]);
        }
    }
    /* ---- reverse P2G ---- */
    for (int64_t p = 0; p < n; ++p) {
        stencil S;
        make_stencil(&x[3 * p], inv_dx, &S);
        double mp = rho * vol[p];
        double k = 4.0 * dt * vol[p] * inv_dx * inv_dx;
        double tau[9], A[9];
        orc_kirchhoff(&mats[p], &F[9 * p], 1.0, tau);
        for (int e = 0; e < 9; ++e)
            A[e] = mp * C[9 * p + e] - k * tau[e];
        double Abar[9] = {0};
        double* xb = &g_in[24 * p];
        double* vb = &g_in[24 * p + 3];
        double* Cb = &g_in[24 * p + 6];
        double* Fb = &g_in[24 * p + 15];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int kk = 0; kk < 3; ++kk) {
                    int64_t id = node_index(&g, &S, i, j, kk);
                    if (id < 0)
                        continue;
                    double wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                    double gw[3] = {inv_dx * S.dw[0][i] * S.w[1][j] * S.w[2][kk],
                                    inv_dx * S.w[0][i] * S.dw[1][j] * S.w[2][kk],
                                    inv_dx * S.w[0][i] * S.w[1][j] * S.dw[2][kk]};
                    double d[3] = {(i - S.f[0]) * h, (j - S.f[1]) * h, (kk - S.f[2]) * h};
                    const double* Pb = &Pbar[3 * id];
                    double contrib = mp * mbar[id];
                    double ATPb[3];
                    for (int a = 0; a < 3; ++a) {
                        double q = mp * v[3 * p + a] + AT(A, a, 0) * d[0] + AT(A, a, 1) * d[1] + AT(A, a, 2) * d[2];
                        contrib += Pb[a] * q;
                        vb[a] += wt * mp * Pb[a];
                        ATPb[a] = AT(A, 0, a) * Pb[0] + AT(A, 1, a) * Pb[1] + AT(A, 2, a) * Pb[2];
                        for (int b = 0; b < 3; ++b)
                            AT(Abar, a, b) += wt * Pb[a] * d[b];
                    }
                    for (int a = 0; a < 3; ++a)
                        xb[a] += gw[a] * contrib - wt * ATPb[a];
                }
        double taubar[9], Ftau[9];
        for (int e = 0; e < 9; ++e) {
            Cb[e] += mp * Abar[e];
            taubar[e] = -k * Abar[e];
        }
        stress_vjp(&mats[p], &F[9 * p], taubar, Ftau);
        for (int e = 0; e < 9; ++e)
            Fb[e] += Ftau[e];
        /* dL/dE through mu and lambda: tau is linear in (mu, lambda) */
        orc_material m1 = elastic(1.0, nu, rho);   /* E = 1: the (mu, lambda) per unit E */
        double t1[9];
        orc_kirchhoff(&m1, &F[9 * p], 1.0, t1);
        double s = 0;
        for (int e = 0; e < 9; ++e)
            s += taubar[e] * t1[e];
        gE[p] += s;
    }
    free(x); free(v); free(C); free(F); free(g.m); free(g.p); free(P); free(mats); free(mat); free(Jp);
    free(vbar_i); free(Pbar); free(mbar);
    return st;
}
