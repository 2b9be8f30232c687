/*
 * Oracle (test infrastructure only): quadratic B-spline weights.
 *
 * The paper uses quadratic B-spline weighting (Sec. 3.1, weight spilling;
 * Sec. 4, 27 nodes per particle).  For a particle at grid coordinate
 * X = x/dx, the base node is floor(X - 0.5) and f = X - base lies in
 * [0.5, 1.5).  The three weights are the quadratic B-spline N(u) evaluated
 * at u = f, f - 1 and f - 2:
 *   N(u) = 3/4 - u^2          for |u| < 1/2
 *   N(u) = (3/2 - |u|)^2 / 2  for 1/2 <= |u| < 3/2
 */
#include "oracle.h"

void orc_bspline_weights(double f, double w[3])
{
    double a = 1.5 - f;      /* |u| for node 0 is f, in [0.5, 1.5) */
    double b = f - 1.0;      /* node 1: |u| < 0.5 */
    double c = f - 0.5;      /* node 2: |u| = 2 - f, 3/2 - |u| = f - 1/2 */
    w[0] = 0.5 * a * a;
    w[1] = 0.75 - b * b;
    w[2] = 0.5 * c * c;
}
