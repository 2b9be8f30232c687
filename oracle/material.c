/*
 * Oracle (test infrastructure only): constitutive models and return maps.
 *
 * The paper merges "singular value decomposition, plasticity projection,
 * stress computation" into the particle kernels (Sec. 4.1) and simulates
 * sand, snow and water (Sec. 6); it prints none of the formulas.  The
 * formulas below are the cited literature's:
 *   fixed-corotated:  tau = 2 mu (F - R) F^T + lambda J (J - 1) I,
 *                     R = U V^T (Stomakhin et al. 2012)
 *   snow:             mu, lambda scaled by exp(xi (1 - Jp)); after the
 *                     F update the singular values are clamped to
 *                     [1 - theta_c, 1 + theta_s] and Jp absorbs the removed
 *                     volume (Stomakhin et al. 2013)
 *   fluid:            tau = -p J I, p = K (J^-gamma - 1)
 *                     (Tampubolon et al. 2017)
 *   sand:             tau = U (2 mu eps + lambda tr(eps) I) U^T with the
 *                     Hencky strain eps = ln(sigma), and the Drucker-Prager
 *                     return map of Klar et al. 2016 (cases I-III).
 *   NACC snow:        the non-associative Cam-Clay model the paper uses for
 *                     its snow scene (Sec. 6.5, parameters kappa, nu, M, beta,
 *                     xi in the notation of Wolper et al. 2019): the same
 *                     Hencky elasticity with mu, lambda from the bulk modulus
 *                     kappa and nu; with p = -tr(tau)/3 and
 *                     q = sqrt(3/2) |dev tau|, the yield surface
 *                     y = (1 + 2 beta) q^2 + M^2 (p + beta p0)(p - p0) = 0,
 *                     p0 = kappa sinh(xi max(-alpha, 0)), alpha = alpha0 + ln Jp;
 *                     the return map keeps p and scales q onto the surface
 *                     (non-associative), or moves to the tips (p0, 0) and
 *                     (-beta p0, 0) beyond them; Jp absorbs the volume the
 *                     projection removes.
 *   neo-Hookean sand: the sand model the paper's sand benchmark uses (Sec. 6,
 *                     after Yue et al. 2018): neo-Hookean elasticity,
 *                     tau = mu (F F^T - I) + lambda ln(J) I, with the same
 *                     Drucker-Prager return map on the Hencky strain as sand.
 * Points the sources leave open: a non-positive singular value is floored at
 * 1e-4 before its logarithm (an inverted sand particle); on the boundaries of
 * the sand return map, tr eps = 0 counts as tension (projected to the apex)
 * and dgamma = 0 as inside the cone (left unchanged).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define AT(M, r, c) (M)[3 * (r) + (c)]
#define ORC_PI 3.14159265358979323846

void orc_lame(double E, double nu, double* mu, double* la)
{
    *mu = E / (2.0 * (1.0 + nu));
    *la = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

static double det3(const double M[9])
{
    return AT(M, 0, 0) * (AT(M, 1, 1) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 1))
         - AT(M, 0, 1) * (AT(M, 1, 0) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 0))
         + AT(M, 0, 2) * (AT(M, 1, 0) * AT(M, 2, 1) - AT(M, 1, 1) * AT(M, 2, 0));
}

/* out = A B^T */
static void mul_abt(const double A[9], const double B[9], double out[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k)
                s += AT(A, i, k) * AT(B, j, k);
            AT(out, i, j) = s;
        }
}

/* out = U diag(d) W^T */
static void udwt(const double U[9], const double d[3], const double W[9], double out[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k)
                s += AT(U, i, k) * d[k] * AT(W, j, k);
            AT(out, i, j) = s;
        }
}

static void fixed_corotated(double mu, double la, const double F[9], double tau[9])
{
    double U[9], sig[3], V[9], R[9], D[9];
    orc_svd3(F, U, sig, V);
    mul_abt(U, V, R);                    /* R = U V^T */
    double J = det3(F);
    for (int i = 0; i < 9; ++i)
        D[i] = F[i] - R[i];
    mul_abt(D, F, tau);                  /* (F - R) F^T */
    for (int i = 0; i < 9; ++i)
        tau[i] *= 2.0 * mu;
    for (int i = 0; i < 3; ++i)
        AT(tau, i, i) += la * J * (J - 1.0);
}

/* Hencky strain of the singular values; a non-positive (inverted) value is
 * read as the floor 1e-4 before the logarithm. */
static void hencky(const double sig[3], double eps[3])
{
    for (int i = 0; i < 3; ++i)
        eps[i] = log(sig[i] > 1e-4 ? sig[i] : 1e-4);
}

/* Lame parameters from the bulk modulus kappa and Poisson ratio nu. */
static void nacc_lame(double kappa, double nu, double* mu, double* la)
{
    *mu = 3.0 * kappa * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu));
    *la = kappa - 2.0 * *mu / 3.0;
}

/* NACC return map on the principal Hencky strains eps (in place).  Returns
 * the change of ln det F (trial minus projected); see the file comment. */
static double nacc_project(const orc_material* mat, double Jp, double eps[3])
{
    double mu, la;
    nacc_lame(mat->E, mat->nu, &mu, &la);
    const double kappa = mat->E, M = mat->friction_M, beta = mat->cohesion;
    double tr = eps[0] + eps[1] + eps[2];
    double dev[3], nd = 0.0;
    for (int i = 0; i < 3; ++i) {
        dev[i] = eps[i] - tr / 3.0;
        nd += dev[i] * dev[i];
    }
    nd = sqrt(nd);
    double p = -kappa * tr;                       /* -tr(tau) / 3 with tr(tau) = 3 kappa tr(eps) */
    double q = sqrt(1.5) * 2.0 * mu * nd;         /* sqrt(3/2) |dev tau|, dev tau = 2 mu dev eps */
    double alpha = mat->alpha0 + log(Jp);
    double p0 = kappa * sinh(mat->hardening * (alpha < 0.0 ? -alpha : 0.0));
    double pn = p, qn = q;
    if (p > p0) {
        pn = p0;
        qn = 0.0;
    } else if (p < -beta * p0) {
        pn = -beta * p0;
        qn = 0.0;
    } else {
        double y = (1.0 + 2.0 * beta) * q * q + M * M * (p + beta * p0) * (p - p0);
        if (y > 0.0)
            qn = sqrt(M * M * (p + beta * p0) * (p0 - p) / (1.0 + 2.0 * beta));
    }
    double trn = -pn / kappa;
    double s = q > 0.0 ? qn / q : 0.0;
    for (int i = 0; i < 3; ++i)
        eps[i] = trn / 3.0 + s * dev[i];
    return tr - trn;
}

void orc_kirchhoff(const orc_material* mat, const double F[9], double Jp, double tau[9])
{
    double mu, la;
    memset(tau, 0, 9 * sizeof(double));
    switch (mat->kind) {
    case ORC_ELASTIC:
        orc_lame(mat->E, mat->nu, &mu, &la);
        fixed_corotated(mu, la, F, tau);
        break;
    case ORC_SNOW: {
        orc_lame(mat->E, mat->nu, &mu, &la);
        double h = exp(mat->hardening * (1.0 - Jp));
        fixed_corotated(mu * h, la * h, F, tau);
        break;
    }
    case ORC_FLUID: {
        double J = Jp;
        double p = mat->E * (pow(J, -mat->gamma) - 1.0);
        for (int i = 0; i < 3; ++i)
            AT(tau, i, i) = -p * J;
        break;
    }
    case ORC_NHSAND: {
        orc_lame(mat->E, mat->nu, &mu, &la);
        const double lnJ = log(det3(F));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double b = 0.0;
                for (int k = 0; k < 3; ++k)
                    b += AT(F, i, k) * AT(F, j, k);
                AT(tau, i, j) = mu * (b - (i == j ? 1.0 : 0.0)) + (i == j ? la * lnJ : 0.0);
            }
        break;
    }
    case ORC_NACC:
    case ORC_SAND: {
        if (mat->kind == ORC_NACC)
            nacc_lame(mat->E, mat->nu, &mu, &la);
        else
            orc_lame(mat->E, mat->nu, &mu, &la);
        double U[9], sig[3], V[9], eps[3], d[3];
        orc_svd3(F, U, sig, V);
        hencky(sig, eps);
        double tr = eps[0] + eps[1] + eps[2];
        for (int i = 0; i < 3; ++i)
            d[i] = 2.0 * mu * eps[i] + la * tr;
        udwt(U, d, U, tau);
        break;
    }
    default:
        break;
    }
}

void orc_plasticity(const orc_material* mat, double F[9], double* Jp)
{
    if (mat->kind == ORC_NACC) {
        double U[9], sig[3], V[9], eps[3], s[3];
        orc_svd3(F, U, sig, V);
        hencky(sig, eps);
        double dlnJ = nacc_project(mat, *Jp, eps);
        for (int i = 0; i < 3; ++i)
            s[i] = exp(eps[i]);
        udwt(U, s, V, F);
        *Jp *= exp(dlnJ);
        return;
    }
    if (mat->kind == ORC_SNOW) {
        double U[9], sig[3], V[9], cl[3];
        orc_svd3(F, U, sig, V);
        double lo = 1.0 - mat->theta_c, hi = 1.0 + mat->theta_s;
        for (int i = 0; i < 3; ++i)
            cl[i] = sig[i] < lo ? lo : (sig[i] > hi ? hi : sig[i]);
        *Jp *= (sig[0] * sig[1] * sig[2]) / (cl[0] * cl[1] * cl[2]);
        udwt(U, cl, V, F);
    } else if (mat->kind == ORC_SAND || mat->kind == ORC_NHSAND) {
        double mu, la;
        orc_lame(mat->E, mat->nu, &mu, &la);
        double U[9], sig[3], V[9], eps[3], s[3];
        orc_svd3(F, U, sig, V);
        hencky(sig, eps);
        double tr = eps[0] + eps[1] + eps[2];
        double sphi = sin(mat->friction_deg * ORC_PI / 180.0);
        double alpha = sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi);
        if (tr >= 0.0) {
            /* case II: expansion, project to the cone tip */
            s[0] = s[1] = s[2] = 1.0;
            udwt(U, s, V, F);
            return;
        }
        double dev[3], nd = 0;
        for (int i = 0; i < 3; ++i) {
            dev[i] = eps[i] - tr / 3.0;
            nd += dev[i] * dev[i];
        }
        nd = sqrt(nd);
        double dgamma = nd + (3.0 * la + 2.0 * mu) / (2.0 * mu) * tr * alpha;
        if (dgamma <= 0.0)
            return; /* case I: inside the yield cone, F unchanged */
        /* case III: radial return onto the cone surface */
        for (int i = 0; i < 3; ++i)
            s[i] = exp(eps[i] - dgamma * dev[i] / nd);
        udwt(U, s, V, F);
    }
}

/* Adaptive step size (the paper's scenes take their step sizes from Fang et
 * al. 2018, Sec. 6.5): dt = min(dt_max, cfl dx / (v + c)), v a bound on the
 * particle speed and c the largest dilatational (p-wave) speed of the
 * materials, c^2 = (lambda + 2 mu) / rho, or K gamma / rho for the fluid
 * p = K (J^-gamma - 1), whose bulk modulus -J dp/dJ at J = 1 is K gamma. */
double orc_wave_speed(const orc_material* mat)
{
    double mu, la;
    if (mat->kind == ORC_FLUID)
        return sqrt(mat->E * mat->gamma / mat->rho);
    if (mat->kind == ORC_NACC)
        nacc_lame(mat->E, mat->nu, &mu, &la);
    else
        orc_lame(mat->E, mat->nu, &mu, &la);
    return sqrt((la + 2.0 * mu) / mat->rho);   /* neo-Hookean: the same at rest */
}

double orc_cfl_dt(const orc_config* cfg, const orc_material* mats, int n_mats, double v_bound, double cfl,
                  double dt_max)
{
    double c = 0.0;
    for (int i = 0; i < n_mats; ++i) {
        double ci = orc_wave_speed(&mats[i]);
        if (ci > c)
            c = ci;
    }
    double dt = cfl * cfg->dx / (v_bound + c);
    return dt < dt_max ? dt : dt_max;
}
