/*
 * vpx_oracle.c -- TEST INFRASTRUCTURE ONLY.  Plain, slow, CPU, FP64.
 *
 * Direct evaluation of the volume potential of a piecewise-polynomial source
 * on the leaves of a quad-tree:
 *
 *     V(x) = (1/2pi) * sum_B  int_B log|x - y| p_B(y) dy            (eq. volinte)
 *
 * where p_B is the tensor-product Lagrange interpolant of the K x K node values
 * of leaf B (Gauss-Legendre nodes).  The near field of a VFMM is exact for this
 * piecewise polynomial (Section 1, Remark after the VFMM definition), so this is
 * the quantity the fast method approximates; here it is computed without any
 * expansion, by quadrature on every (target, leaf) pair:
 *
 *  - well separated leaves (distance >= side): tensor Gauss-Legendre, the
 *    order chosen from the distance/side ratio;
 *  - near and self leaves: singularity subtraction at the point x* of B
 *    closest to x,
 *        int_B log|x-y| l_j(y) dy = l_j(x*) J_B(x)
 *                                 + int_B log|x-y| (l_j(y) - l_j(x*)) dy,
 *    with J_B(x) = int_B log|x-y| dy in closed form and the (continuous)
 *    remainder integrated on B split at x* into rectangles that are graded
 *    dyadically toward x*.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may call
 * this file.  It shares no code with the CUDA library.
 *
 * Node ordering of a leaf: node (a, b) -> index b*K + a, x from t[a], y from t[b],
 * t the K Gauss-Legendre nodes of [-1, 1] in ascending order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- GL rules */

/* n-point Gauss-Legendre rule on [-1,1], ascending nodes (Newton iteration on
 * the three-term recurrence of the Legendre polynomials). */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        /* initial guess for the i-th largest root */
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                /* one more step for full accuracy */
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ---------------------------------------------------------- Lagrange basis */

/* values of the K Lagrange basis polynomials for nodes t[] at point s */
static void lagrange_values(int K, const double *t, double s, double *out)
{
    for (int a = 0; a < K; ++a) {
        double v = 1.0;
        for (int m = 0; m < K; ++m)
            if (m != a) v *= (s - t[m]) / (t[a] - t[m]);
        out[a] = v;
    }
}

/* ------------------------------------------------------ closed-form J_B(x) */

/* G(u,v) = int_0^u int_0^v log(s^2 + t^2) dt ds
 *        = u v (log(u^2+v^2) - 3) + u^2 atan(v/u) + v^2 atan(u/v),
 * with the limits G(0,v) = G(u,0) = 0. */
static double Gcorner(double u, double v)
{
    if (u == 0.0 || v == 0.0) return 0.0;
    return u * v * (log(u * u + v * v) - 3.0) + u * u * atan(v / u) + v * v * atan(u / v);
}

/* J = int over [x0,x1]x[y0,y1] of log|x - y| dy, target (px, py) */
double orc_rect_log_integral(double px, double py, double x0, double x1, double y0, double y1)
{
    double u0 = x0 - px, u1 = x1 - px, v0 = y0 - py, v1 = y1 - py;
    return 0.5 * (Gcorner(u1, v1) - Gcorner(u0, v1) - Gcorner(u1, v0) + Gcorner(u0, v0));
}

/* ------------------------------------------------ per-leaf basis integrals */

typedef struct {
    int K;
    const double *t;      /* K leaf nodes on [-1,1] */
    int Q;                /* order for graded pieces */
    const double *gq, *gw;/* Q-point GL on [-1,1] */
} near_ctx;

/* Accumulate over rectangle R = [ux0,ux1] x [uy0,uy1] (physical coords) with a
 * Q x Q tensor GL rule:
 *     I[b*K+a] += sum w log|x-y| l_a(y1') l_b(y2')      (y' = leaf reference coords)
 *     *S       += sum w log|x-y|
 */
static void accumulate_rect(const near_ctx *c, double px, double py,
                            double cx, double cy, double h,
                            double ux0, double ux1, double uy0, double uy1,
                            double *I, double *S)
{
    const int K = c->K, Q = c->Q;
    double la[32 * 32], lb[32 * 32];   /* [i][a] basis at the Q abscissae */
    double yq[64], xq[64], wx[64], wy[64];
    double hx = 0.5 * (ux1 - ux0), hy = 0.5 * (uy1 - uy0);
    double mx = 0.5 * (ux1 + ux0), my = 0.5 * (uy1 + uy0);
    for (int i = 0; i < Q; ++i) {
        xq[i] = mx + hx * c->gq[i];
        yq[i] = my + hy * c->gq[i];
        wx[i] = hx * c->gw[i];
        wy[i] = hy * c->gw[i];
        lagrange_values(K, c->t, (xq[i] - cx) / h, la + i * K);
        lagrange_values(K, c->t, (yq[i] - cy) / h, lb + i * K);
    }
    double M[64 * 32];  /* M[i][b] = sum_j wy_j log|x - y_ij| l_b(y_j) */
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
        for (int b = 0; b < K; ++b) M[i * K + b] = 0.0;
        double dx = xq[i] - px;
        for (int j = 0; j < Q; ++j) {
            double dy = yq[j] - py;
            double g = 0.5 * log(dx * dx + dy * dy) * wy[j];
            s += g * wx[i];
            for (int b = 0; b < K; ++b) M[i * K + b] += g * lb[j * K + b];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int b = 0; b < K; ++b) {
            double m = M[i * K + b] * wx[i];
            for (int a = 0; a < K; ++a) I[b * K + a] += m * la[i * K + a];
        }
    *S += s;
}

/* Rectangle with the (near-)singular point at one corner (sx, sy); the
 * rectangle extends by ex (signed) in x and ey (signed) in y.  Elongated
 * rectangles are first cut into geometrically growing strips; the square-ish
 * corner part is graded dyadically toward the corner (L-shaped layers). */
static void corner_rect(const near_ctx *c, double px, double py, double cx, double cy, double h,
                        double sx, double sy, double ex, double ey, double *I, double *S)
{
    double ax = fabs(ex), ay = fabs(ey);
    if (ax == 0.0 || ay == 0.0) return;
    double dxs = ex > 0 ? 1.0 : -1.0, dys = ey > 0 ? 1.0 : -1.0;
    /* strips along the long side */
    if (ax > 2.0 * ay) {
        double u0 = ay;
        while (u0 < ax) {
            double u1 = fmin(2.0 * u0, ax);
            if (ax - u1 < 0.5 * u0) u1 = ax;
            double X0 = sx + dxs * u0, X1 = sx + dxs * u1;
            double Y0 = sy, Y1 = sy + dys * ay;
            accumulate_rect(c, px, py, cx, cy, h, fmin(X0, X1), fmax(X0, X1), fmin(Y0, Y1), fmax(Y0, Y1), I, S);
            u0 = u1;
        }
        ax = ay;
    } else if (ay > 2.0 * ax) {
        double v0 = ax;
        while (v0 < ay) {
            double v1 = fmin(2.0 * v0, ay);
            if (ay - v1 < 0.5 * v0) v1 = ay;
            double Y0 = sy + dys * v0, Y1 = sy + dys * v1;
            double X0 = sx, X1 = sx + dxs * ax;
            accumulate_rect(c, px, py, cx, cy, h, fmin(X0, X1), fmax(X0, X1), fmin(Y0, Y1), fmax(Y0, Y1), I, S);
            v0 = v1;
        }
        ay = ax;
    }
    /* dyadic layers toward the corner, stop below 1e-6 of the leaf side */
    double stop = 2e-6 * h;
    while (fmax(ax, ay) > stop) {
        double bx = 0.5 * ax, by = 0.5 * ay;
        double r[3][4] = {
            {bx, ax, 0.0, by},
            {0.0, bx, by, ay},
            {bx, ax, by, ay},
        };
        for (int k = 0; k < 3; ++k) {
            double X0 = sx + dxs * r[k][0], X1 = sx + dxs * r[k][1];
            double Y0 = sy + dys * r[k][2], Y1 = sy + dys * r[k][3];
            accumulate_rect(c, px, py, cx, cy, h, fmin(X0, X1), fmax(X0, X1), fmin(Y0, Y1), fmax(Y0, Y1), I, S);
        }
        ax = bx;
        ay = by;
    }
}

/* Basis integrals for a near/self leaf: I[j] = int_B log|x-y| l_j(y) dy. */
static void near_leaf_basis_integrals(const near_ctx *c, double px, double py,
                                      double cx, double cy, double h, double *I)
{
    const int K = c->K;
    double x0 = cx - h, x1 = cx + h, y0 = cy - h, y1 = cy + h;
    double qx = fmin(fmax(px, x0), x1), qy = fmin(fmax(py, y0), y1);  /* x* */
    double Rem[32 * 32];
    for (int j = 0; j < K * K; ++j) Rem[j] = 0.0;
    double S = 0.0;
    /* B split at x* into up to four rectangles with corner x* */
    corner_rect(c, px, py, cx, cy, h, qx, qy, x1 - qx, y1 - qy, Rem, &S);
    corner_rect(c, px, py, cx, cy, h, qx, qy, x0 - qx, y1 - qy, Rem, &S);
    corner_rect(c, px, py, cx, cy, h, qx, qy, x1 - qx, y0 - qy, Rem, &S);
    corner_rect(c, px, py, cx, cy, h, qx, qy, x0 - qx, y0 - qy, Rem, &S);
    double J = orc_rect_log_integral(px, py, x0, x1, y0, y1);
    double lqa[32], lqb[32];
    lagrange_values(K, c->t, (qx - cx) / h, lqa);
    lagrange_values(K, c->t, (qy - cy) / h, lqb);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) {
            double lstar = lqa[a] * lqb[b];
            I[b * K + a] = lstar * J + (Rem[b * K + a] - lstar * S);
        }
}

/* Exported for tests: basis integrals of one leaf at one target, choosing the
 * near or far rule exactly as the potential routine does. */
void orc_leaf_basis_integrals(int K, const double *t, double cx, double cy, double h,
                              double px, double py, double *I);

/* ------------------------------------------------------- far-field rules */

typedef struct {
    int Q;
    double g[32], w[32];
    double L[32 * 32];   /* L[i][a] = l_a(g_i) */
} far_rule;

static void far_rule_init(far_rule *r, int Q, int K, const double *t)
{
    r->Q = Q;
    orc_gauss_legendre(Q, r->g, r->w);
    for (int i = 0; i < Q; ++i) lagrange_values(K, t, r->g[i], r->L + i * K);
}

/* order of the tensor GL rule for a leaf at distance d, side s (d >= s) */
static int far_order_index(double d, double s)
{
    if (d >= 4.0 * s) return 2;
    if (d >= 2.0 * s) return 1;
    return 0;
}

static double box_distance(double px, double py, double cx, double cy, double h)
{
    double dx = fabs(px - cx) - h, dy = fabs(py - cy) - h;
    dx = dx > 0 ? dx : 0.0;
    dy = dy > 0 ? dy : 0.0;
    return sqrt(dx * dx + dy * dy);
}

/* The integrand is a basis polynomial of degree K-1 per variable times the
 * log kernel; the rules below integrate the kernel part to ~1e-17 and are
 * raised by K/2 points so that the polynomial factor is integrated exactly. */
static const int FAR_Q_BASE[3] = {20, 14, 10};
static int far_q(int qi, int K) { return FAR_Q_BASE[qi] + K / 2; }
static const int NEAR_Q = 20;

void orc_leaf_basis_integrals(int K, const double *t, double cx, double cy, double h,
                              double px, double py, double *I)
{
    double d = box_distance(px, py, cx, cy, h);
    if (d >= 2.0 * h) {
        far_rule fr;
        far_rule_init(&fr, far_q(far_order_index(d, 2.0 * h), K), K, t);
        for (int j = 0; j < K * K; ++j) I[j] = 0.0;
        for (int i = 0; i < fr.Q; ++i)
            for (int jj = 0; jj < fr.Q; ++jj) {
                double dx = cx + h * fr.g[i] - px, dy = cy + h * fr.g[jj] - py;
                double g = 0.5 * log(dx * dx + dy * dy) * fr.w[i] * fr.w[jj] * h * h;
                for (int b = 0; b < K; ++b)
                    for (int a = 0; a < K; ++a) I[b * K + a] += g * fr.L[i * K + a] * fr.L[jj * K + b];
            }
        return;
    }
    near_ctx c;
    double gq[64], gw[64];
    orc_gauss_legendre(NEAR_Q, gq, gw);
    c.K = K; c.t = t; c.Q = NEAR_Q; c.gq = gq; c.gw = gw;
    near_leaf_basis_integrals(&c, px, py, cx, cy, h, I);
}

/* ---------------------------------------------------------- the potential */

/*
 * V[i*nrhs + r] = (1/2pi) sum_B int_B log|x_i - y| p_{B,r}(y) dy
 *
 * leaf arrays: centre (cx, cy), half side h; values f[(B*nrhs + r)*K*K + j].
 * Leaves whose values are all zero are skipped (they contribute nothing).
 * t: the K leaf nodes on [-1,1].  Returns 0.
 */
int orc_volume_potential(int n_leaves, const double *lcx, const double *lcy, const double *lh,
                         int K, const double *t, int nrhs, const double *f,
                         int n_targets, const double *tx, const double *ty,
                         double *V, int nthreads)
{
    const int KK = K * K;
    if (K > 32 || nrhs > 256) return -1;
    far_rule fr[3];
    for (int q = 0; q < 3; ++q) far_rule_init(&fr[q], far_q(q, K), K, t);
    /* per leaf and rhs: values of p_B at the three far rules' tensor points */
    size_t per = 0;
    for (int q = 0; q < 3; ++q) per += (size_t)far_q(q, K) * far_q(q, K);
    double *P = (double *)malloc(sizeof(double) * per * (size_t)n_leaves * nrhs);
    unsigned char *nz = (unsigned char *)malloc(n_leaves);
    if (!P || !nz) { free(P); free(nz); return -2; }
    for (int B = 0; B < n_leaves; ++B) {
        int any = 0;
        for (int r = 0; r < nrhs; ++r) {
            const double *F = f + ((size_t)B * nrhs + r) * KK;
            for (int j = 0; j < KK; ++j) if (F[j] != 0.0) any = 1;
            double *dst = P + ((size_t)B * nrhs + r) * per;
            for (int q = 0; q < 3; ++q) {
                int Q = far_q(q, K);
                for (int i = 0; i < Q; ++i)
                    for (int jj = 0; jj < Q; ++jj) {
                        double s = 0.0;
                        for (int b = 0; b < K; ++b)
                            for (int a = 0; a < K; ++a)
                                s += F[b * K + a] * fr[q].L[i * K + a] * fr[q].L[jj * K + b];
                        dst[i * Q + jj] = s;
                    }
                dst += (size_t)Q * Q;
            }
        }
        nz[B] = (unsigned char)any;
    }
    double gq[64], gw[64];
    orc_gauss_legendre(NEAR_Q, gq, gw);

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int it = 0; it < n_targets; ++it) {
        near_ctx c;
        c.K = K; c.t = t; c.Q = NEAR_Q; c.gq = gq; c.gw = gw;
        double px = tx[it], py = ty[it];
        double acc[256];
        double I[32 * 32];
        for (int r = 0; r < nrhs && r < 256; ++r) acc[r] = 0.0;
        for (int B = 0; B < n_leaves; ++B) {
            if (!nz[B]) continue;
            double cx = lcx[B], cy = lcy[B], h = lh[B];
            double d = box_distance(px, py, cx, cy, h);
            if (d >= 2.0 * h) {
                int qi = far_order_index(d, 2.0 * h);
                int Q = far_q(qi, K);
                size_t off = 0;
                for (int q = 0; q < qi; ++q) off += (size_t)far_q(q, K) * far_q(q, K);
                for (int r = 0; r < nrhs; ++r) {
                    const double *Pv = P + ((size_t)B * nrhs + r) * per + off;
                    double s = 0.0;
                    for (int i = 0; i < Q; ++i) {
                        double dx = cx + h * fr[qi].g[i] - px;
                        double si = 0.0;
                        for (int jj = 0; jj < Q; ++jj) {
                            double dy = cy + h * fr[qi].g[jj] - py;
                            si += fr[qi].w[jj] * 0.5 * log(dx * dx + dy * dy) * Pv[i * Q + jj];
                        }
                        s += fr[qi].w[i] * si;
                    }
                    acc[r] += s * h * h;
                }
            } else {
                near_leaf_basis_integrals(&c, px, py, cx, cy, h, I);
                for (int r = 0; r < nrhs; ++r) {
                    const double *F = f + ((size_t)B * nrhs + r) * KK;
                    double s = 0.0;
                    for (int j = 0; j < KK; ++j) s += F[j] * I[j];
                    acc[r] += s;
                }
            }
        }
        for (int r = 0; r < nrhs; ++r) V[(size_t)it * nrhs + r] = acc[r] / (2.0 * ORC_PI);
    }
    free(P);
    free(nz);
    return 0;
}

/* number of threads OpenMP will use */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
