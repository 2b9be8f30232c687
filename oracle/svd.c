/*
 * Oracle (test infrastructure only): 3x3 singular value decomposition.
 *
 * The paper names the SVD as one of the per-particle computations merged
 * into the transfer kernels (Sec. 4.1) but does not specify it.  The oracle
 * uses the one-sided (Hestenes) Jacobi method in FP64: rotate pairs of
 * columns of A = F until they are mutually orthogonal, accumulating the
 * rotations in V; then sigma_i = |A e_i| and U e_i = A e_i / sigma_i.
 * Sweeps run until every column pair is orthogonal to 1e-15 relative.
 *
 * Convention (shared with the GPU path only through this statement):
 * sig[0] >= sig[1] >= |sig[2]|, det U = det V = +1, and sig[2] takes the
 * sign of det F (the "rotation-variant" SVD of Irving et al. 2004).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define AT(M, r, c) (M)[3 * (r) + (c)]

static double det3(const double M[9])
{
    return AT(M, 0, 0) * (AT(M, 1, 1) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 1))
         - AT(M, 0, 1) * (AT(M, 1, 0) * AT(M, 2, 2) - AT(M, 1, 2) * AT(M, 2, 0))
         + AT(M, 0, 2) * (AT(M, 1, 0) * AT(M, 2, 1) - AT(M, 1, 1) * AT(M, 2, 0));
}

static void swap_cols(double M[9], int a, int b)
{
    for (int r = 0; r < 3; ++r) {
        double t = AT(M, r, a);
        AT(M, r, a) = AT(M, r, b);
        AT(M, r, b) = t;
    }
}

void orc_svd3(const double F[9], double U[9], double sig[3], double V[9])
{
    double A[9];
    memcpy(A, F, sizeof(A));
    memset(V, 0, 9 * sizeof(double));
    AT(V, 0, 0) = AT(V, 1, 1) = AT(V, 2, 2) = 1.0;

    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k];
            double alpha = 0, beta = 0, gamma = 0;
            for (int r = 0; r < 3; ++r) {
                alpha += AT(A, r, p) * AT(A, r, p);
                beta += AT(A, r, q) * AT(A, r, q);
                gamma += AT(A, r, p) * AT(A, r, q);
            }
            if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta))
                continue;
            rotated = 1;
            /* Rotation (c, s) acting as a_p' = c a_p - s a_q,
             * a_q' = s a_p + c a_q makes a_p' . a_q' = 0 when
             * t = s/c solves t^2 + 2 zeta t - 1 = 0; take the smaller root. */
            double zeta = (beta - alpha) / (2.0 * gamma);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t);
            double s = c * t;
            for (int r = 0; r < 3; ++r) {
                double ap = AT(A, r, p), aq = AT(A, r, q);
                AT(A, r, p) = c * ap - s * aq;
                AT(A, r, q) = s * ap + c * aq;
                double vp = AT(V, r, p), vq = AT(V, r, q);
                AT(V, r, p) = c * vp - s * vq;
                AT(V, r, q) = s * vp + c * vq;
            }
        }
        if (!rotated)
            break;
    }

    for (int i = 0; i < 3; ++i)
        sig[i] = sqrt(AT(A, 0, i) * AT(A, 0, i) + AT(A, 1, i) * AT(A, 1, i) + AT(A, 2, i) * AT(A, 2, i));

    /* sort descending (selection sort on three entries) */
    for (int i = 0; i < 2; ++i) {
        int m = i;
        for (int j = i + 1; j < 3; ++j)
            if (sig[j] > sig[m])
                m = j;
        if (m != i) {
            double t = sig[i];
            sig[i] = sig[m];
            sig[m] = t;
            swap_cols(A, i, m);
            swap_cols(V, i, m);
        }
    }

    /* U columns: normalised A columns; rank-deficient columns are
     * completed to an orthonormal basis. */
    double scale = sig[0] > 0 ? sig[0] : 1.0;
    for (int i = 0; i < 3; ++i) {
        if (sig[i] > 1e-300 && sig[i] > 1e-14 * scale) {
            for (int r = 0; r < 3; ++r)
                AT(U, r, i) = AT(A, r, i) / sig[i];
        } else if (i == 0) {
            AT(U, 0, 0) = 1; AT(U, 1, 0) = 0; AT(U, 2, 0) = 0;
        } else if (i == 1) {
            /* any unit vector orthogonal to u0 */
            double u0[3] = {AT(U, 0, 0), AT(U, 1, 0), AT(U, 2, 0)};
            double e[3] = {0, 0, 0};
            int small = 0;
            for (int r = 1; r < 3; ++r)
                if (fabs(u0[r]) < fabs(u0[small]))
                    small = r;
            e[small] = 1.0;
            double d = e[0] * u0[0] + e[1] * u0[1] + e[2] * u0[2];
            double w[3], nw = 0;
            for (int r = 0; r < 3; ++r) {
                w[r] = e[r] - d * u0[r];
                nw += w[r] * w[r];
            }
            nw = sqrt(nw);
            for (int r = 0; r < 3; ++r)
                AT(U, r, 1) = w[r] / nw;
        } else {
            /* u2 = u0 x u1 */
            AT(U, 0, 2) = AT(U, 1, 0) * AT(U, 2, 1) - AT(U, 2, 0) * AT(U, 1, 1);
            AT(U, 1, 2) = AT(U, 2, 0) * AT(U, 0, 1) - AT(U, 0, 0) * AT(U, 2, 1);
            AT(U, 2, 2) = AT(U, 0, 0) * AT(U, 1, 1) - AT(U, 1, 0) * AT(U, 0, 1);
        }
    }

    /* Make both factors proper rotations, moving the sign into sig[2]:
     * flipping column 2 of V (or of U) flips the sign of the rank-one
     * term u2 sig2 v2^T, which is compensated by negating sig[2]. */
    if (det3(V) < 0) {
        for (int r = 0; r < 3; ++r)
            AT(V, r, 2) = -AT(V, r, 2);
        sig[2] = -sig[2];
    }
    if (det3(U) < 0) {
        for (int r = 0; r < 3; ++r)
            AT(U, r, 2) = -AT(U, r, 2);
        sig[2] = -sig[2];
    }
}
