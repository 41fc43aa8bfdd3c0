/*
 * fem_oracle.c -- plain FP64 CPU oracle for the element-local tensor-product
 * matvecs BP1.0, BP3.5 and BP3.0 of Swirydowicz, Chalmers, Karakus and
 * Warburton, "Acceleration of tensor-product operations for high-order finite
 * element methods" (arXiv:1711.00903).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code, header
 * or table with the CUDA library: nodes, weights, operator matrices and
 * geometric factors are all recomputed here from their definitions.
 *
 * Everything is IEEE double, no fast-math, no blocking or fusion beyond the
 * sum factorisation the paper states.  Index conventions (0-based):
 *   n = N+1 GLL points per direction, m = N+2 Gauss points per direction;
 *   node (i,j,k) of an element is stored at i + n*j + n*n*k (i = r fastest);
 *   I is m x n row-major (I[a*n+i] = l_i(rt_a));
 *   D is n x n (D[a*n+i] = l_i'(r_a)); Dt is m x m (Dt[a*m+b] = lt_b'(rt_a));
 *   geometric factors are stored per element as 7 planes of nodes:
 *   geo[(e*7 + g)*npts + node], g = Grr, Grs, Grt, Gss, Gst, Gtt, wJ
 *   (BP1.0 stores the wJ plane alone: geo[e*npts + node]).
 *   Vertices: verts[(e*8 + c)*3 + d], corner c = cr + 2cs + 4ct with
 *   cr, cs, ct in {0,1} meaning r, s, t = -1 or +1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXN 15
#define OR_MAXQ (OR_MAXN + 2)

/* ------------------------------------------------------------------ */
/* Threads                                                             */
/* ------------------------------------------------------------------ */

int or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* 1D quadrature (Section 4: GLL nodes r_i, weights w_i, N+1 points;  */
/* Gauss-Legendre nodes rt_a, weights wt_a, N+2 points)               */
/* ------------------------------------------------------------------ */

/* Legendre P_k(x) for k = p (returned) and p-1 (*pm1) by Bonnet's
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static double legendre(int p, double x, double *pm1)
{
    double a = 1.0, b = x; /* P_0, P_1 */
    if (p == 0) { if (pm1) *pm1 = 0.0; return 1.0; }
    for (int k = 1; k < p; k++) {
        double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = c;
    }
    if (pm1) *pm1 = a;
    return b;
}

/* P_p'(x) for |x| < 1 from (1 - x^2) P_p' = p (P_{p-1} - x P_p). */
static double legendre_d1(int p, double x, double *P)
{
    double pm1, pp = legendre(p, x, &pm1);
    if (P) *P = pp;
    return p * (pm1 - x * pp) / (1.0 - x * x);
}

/* m-point Gauss-Legendre rule: the nodes are the roots of P_m, found by
 * Newton's method from the Chebyshev-type guesses cos(pi (j + 3/4)/(m + 1/2));
 * weights 2 / ((1 - x^2) P_m'(x)^2).  Nodes ascend. */
int or_gauss(int m, double *x, double *w)
{
    if (m < 1 || m > 64) return -1;
    for (int j = 0; j < m; j++) {
        double xi = -cos(M_PI * (j + 0.75) / (m + 0.5));
        for (int it = 0; it < 100; it++) {
            double P, dP = legendre_d1(m, xi, &P);
            double dx = P / dP;
            xi -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        x[j] = xi;
    }
    for (int j = 0; j < m / 2; j++) { /* exact mirror symmetry */
        double s = 0.5 * (x[m - 1 - j] - x[j]);
        x[j] = -s;
        x[m - 1 - j] = s;
    }
    if (m % 2) x[m / 2] = 0.0;
    for (int j = 0; j < m; j++) {
        double dP = legendre_d1(m, x[j], NULL);
        w[j] = 2.0 / ((1.0 - x[j] * x[j]) * dP * dP);
    }
    return 0;
}

/* N+1 point Gauss-Lobatto-Legendre rule: -1, +1 and the roots of P_N',
 * found by Newton's method on P_N' (P_N'' from Legendre's equation
 * (1 - x^2) P'' = 2 x P' - N(N+1) P) from the Chebyshev-Gauss-Lobatto
 * guesses -cos(pi j / N); weights 2 / (N (N+1) P_N(x)^2).  Nodes ascend. */
int or_gll(int N, double *x, double *w)
{
    if (N < 1 || N > 64) return -1;
    int n = N + 1;
    x[0] = -1.0;
    x[N] = 1.0;
    for (int j = 1; j < N; j++) {
        double xi = -cos(M_PI * j / N);
        for (int it = 0; it < 100; it++) {
            double P, d1 = legendre_d1(N, xi, &P);
            double d2 = (2.0 * xi * d1 - N * (N + 1.0) * P) / (1.0 - xi * xi);
            double dx = d1 / d2;
            xi -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        x[j] = xi;
    }
    for (int j = 0; j < n / 2; j++) {
        double s = 0.5 * (x[n - 1 - j] - x[j]);
        x[j] = -s;
        x[n - 1 - j] = s;
    }
    if (n % 2) x[n / 2] = 0.0;
    for (int j = 0; j < n; j++) {
        double P = legendre(N, x[j], NULL);
        w[j] = 2.0 / (N * (N + 1.0) * P * P);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Lagrange basis on a node set, by the product formula               */
/* ------------------------------------------------------------------ */

/* l_i(x) = prod_{k != i} (x - x_k) / (x_i - x_k) */
static double lagrange(int n, const double *xn, int i, double x)
{
    double v = 1.0;
    for (int k = 0; k < n; k++)
        if (k != i) v *= (x - xn[k]) / (xn[i] - xn[k]);
    return v;
}

/* l_i'(x) = sum_{j != i} 1/(x_i - x_j) prod_{k != i, j} (x - x_k)/(x_i - x_k)
 * (product rule applied to the product formula) */
static double lagrange_d1(int n, const double *xn, int i, double x)
{
    double s = 0.0;
    for (int j = 0; j < n; j++) {
        if (j == i) continue;
        double t = 1.0 / (xn[i] - xn[j]);
        for (int k = 0; k < n; k++)
            if (k != i && k != j) t *= (x - xn[k]) / (xn[i] - xn[k]);
        s += t;
    }
    return s;
}

/* Values l_i(x) for every i (used by the tests to evaluate fields). */
void or_lagrange_row(int n, const double *xn, double x, double *out)
{
    for (int i = 0; i < n; i++) out[i] = lagrange(n, xn, i, x);
}

void or_lagrange_d1_row(int n, const double *xn, double x, double *out)
{
    for (int i = 0; i < n; i++) out[i] = lagrange_d1(n, xn, i, x);
}

/* Basis of degree N (Table of notation; eq. interpolationOps; eq.
 * derivativeOps with the derivative the text omits):
 *   r, w   : n GLL nodes / weights       rt, wt : m Gauss nodes / weights
 *   I      : m x n, I[a][i] = l_i(rt_a)
 *   D      : n x n, D[a][i] = l_i'(r_a)
 *   Dt     : m x m, Dt[a][b] = lt_b'(rt_a)  (lt = Lagrange basis on Gauss nodes)
 * Any output pointer may be NULL. */
int or_basis(int N, double *r, double *w, double *rt, double *wt,
             double *I, double *D, double *Dt)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1, m = N + 2;
    double gr[OR_MAXQ], gw[OR_MAXQ], qr[OR_MAXQ], qw[OR_MAXQ];
    or_gll(N, gr, gw);
    or_gauss(m, qr, qw);
    if (r) memcpy(r, gr, n * sizeof(double));
    if (w) memcpy(w, gw, n * sizeof(double));
    if (rt) memcpy(rt, qr, m * sizeof(double));
    if (wt) memcpy(wt, qw, m * sizeof(double));
    if (I)
        for (int a = 0; a < m; a++)
            for (int i = 0; i < n; i++) I[a * n + i] = lagrange(n, gr, i, qr[a]);
    if (D)
        for (int a = 0; a < n; a++)
            for (int i = 0; i < n; i++) D[a * n + i] = lagrange_d1(n, gr, i, gr[a]);
    if (Dt)
        for (int a = 0; a < m; a++)
            for (int b = 0; b < m; b++) Dt[a * m + b] = lagrange_d1(m, qr, b, qr[a]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Geometry (Section 4: trilinear map of the bi-unit cube)            */
/* ------------------------------------------------------------------ */

/* Trilinear map x(r,s,t) = sum_c x_c phi_c with
 * phi_c = (1 + sr r)(1 + ss s)(1 + st t) / 8, and its Jacobian matrix
 * X[d][rho] = d x_d / d rho (rho = r, s, t). */
void or_map(const double *v, double r, double s, double t, double *x, double *X)
{
    for (int d = 0; d < 3; d++) {
        if (x) x[d] = 0.0;
        if (X) X[d * 3 + 0] = X[d * 3 + 1] = X[d * 3 + 2] = 0.0;
    }
    for (int c = 0; c < 8; c++) {
        double sr = (c & 1) ? 1.0 : -1.0;
        double ss = (c & 2) ? 1.0 : -1.0;
        double st = (c & 4) ? 1.0 : -1.0;
        double fr = 1.0 + sr * r, fs = 1.0 + ss * s, ft = 1.0 + st * t;
        for (int d = 0; d < 3; d++) {
            double xc = v[c * 3 + d];
            if (x) x[d] += xc * fr * fs * ft / 8.0;
            if (X) {
                X[d * 3 + 0] += xc * sr * fs * ft / 8.0;
                X[d * 3 + 1] += xc * fr * ss * ft / 8.0;
                X[d * 3 + 2] += xc * fr * fs * st / 8.0;
            }
        }
    }
}

/* At one point: detJ = det X and the scaled metric
 * G = detJ X^{-1} X^{-T}  (G[rho][sigma] = detJ sum_d dr_rho/dx_d dr_sigma/dx_d),
 * the matrix the weak form carries after mapping to the reference cube
 * (Section 4; the text's "|J| J^T J" is read with J the inverse map's
 * Jacobian).  X^{-1} by the adjugate. */
static double metric_at(const double *v, double r, double s, double t, double G[3][3])
{
    double X[9];
    or_map(v, r, s, t, NULL, X);
    double a = X[0], b = X[1], c = X[2];
    double d = X[3], e = X[4], f = X[5];
    double g = X[6], h = X[7], k = X[8];
    double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
    /* inverse = adj / det; adj[i][j] = cofactor[j][i] */
    double inv[3][3];
    inv[0][0] = (e * k - f * h) / det;
    inv[0][1] = -(b * k - c * h) / det;
    inv[0][2] = (b * f - c * e) / det;
    inv[1][0] = -(d * k - f * g) / det;
    inv[1][1] = (a * k - c * g) / det;
    inv[1][2] = -(a * f - c * d) / det;
    inv[2][0] = (d * h - e * g) / det;
    inv[2][1] = -(a * h - b * g) / det;
    inv[2][2] = (a * e - b * d) / det;
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) {
            double sum = 0.0;
            for (int dd = 0; dd < 3; dd++) sum += inv[p][dd] * inv[q][dd];
            G[p][q] = det * sum;
        }
    return det;
}

/* Geometric factors on a tensor grid of q points per direction with 1D
 * nodes x and weights w (GLL for BP3.5, Gauss for BP1.0 and BP3.0):
 *   G_{rr} ... G_{tt} times w_a w_b w_c, and wJ = w_a w_b w_c detJ
 * (the diagonal matrices G^e and J^e of Section 4).
 * kind 1: wJ only (E x q^3); kind 2/3: 7 planes (E x 7 x q^3).
 * Returns the minimum detJ seen (negative means an inverted element). */
double or_geofacs_grid(int q, const double *x, const double *w, int kind,
                       int64_t E, const double *verts, double *geo)
{
    int64_t npts = (int64_t)q * q * q;
    double mindet = INFINITY;
#pragma omp parallel for reduction(min : mindet) schedule(static)
    for (int64_t e = 0; e < E; e++) {
        const double *v = verts + e * 24;
        for (int c = 0; c < q; c++)
            for (int b = 0; b < q; b++)
                for (int a = 0; a < q; a++) {
                    double G[3][3];
                    double det = metric_at(v, x[a], x[b], x[c], G);
                    double W = w[a] * w[b] * w[c];
                    int64_t node = a + (int64_t)q * (b + (int64_t)q * c);
                    if (det < mindet) mindet = det;
                    if (kind == 1) {
                        geo[e * npts + node] = W * det;
                    } else {
                        double *g = geo + e * 7 * npts + node;
                        g[0 * npts] = W * G[0][0];
                        g[1 * npts] = W * G[0][1];
                        g[2 * npts] = W * G[0][2];
                        g[3 * npts] = W * G[1][1];
                        g[4 * npts] = W * G[1][2];
                        g[5 * npts] = W * G[2][2];
                        g[6 * npts] = W * det;
                    }
                }
    }
    return mindet;
}

/* kind 1 = BP1.0 (wJ at Gauss points), 2 = BP3.5 (7 factors at GLL nodes),
 * 3 = BP3.0 (7 factors at Gauss points). */
double or_geofacs(int N, int kind, int64_t E, const double *verts, double *geo)
{
    double r[OR_MAXQ], w[OR_MAXQ], rt[OR_MAXQ], wt[OR_MAXQ];
    if (or_basis(N, r, w, rt, wt, NULL, NULL, NULL)) return NAN;
    if (kind == 2) return or_geofacs_grid(N + 1, r, w, 2, E, verts, geo);
    return or_geofacs_grid(N + 2, rt, wt, kind, E, verts, geo);
}

/* ------------------------------------------------------------------ */
/* Sum-factorised operators (Algorithms 1-5)                          */
/* ------------------------------------------------------------------ */

/* Interpolation GLL -> Gauss (Algorithm 1, read as three 1D contractions,
 * one per direction; no Jacobian scaling inside):
 *   t1[k][j][a] = sum_i I[a][i] q[k][j][i]
 *   t2[k][b][a] = sum_j I[b][j] t1[k][j][a]
 *   qg[c][b][a] = sum_k I[c][k] t2[k][b][a]  */
static void interpolate(int n, int m, const double *I, const double *q, double *qg,
                        double *t1, double *t2)
{
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int a = 0; a < m; a++) {
                double s = 0.0;
                for (int i = 0; i < n; i++) s += I[a * n + i] * q[i + n * (j + n * k)];
                t1[a + m * (j + n * k)] = s;
            }
    for (int k = 0; k < n; k++)
        for (int b = 0; b < m; b++)
            for (int a = 0; a < m; a++) {
                double s = 0.0;
                for (int j = 0; j < n; j++) s += I[b * n + j] * t1[a + m * (j + n * k)];
                t2[a + m * (b + m * k)] = s;
            }
    for (int c = 0; c < m; c++)
        for (int b = 0; b < m; b++)
            for (int a = 0; a < m; a++) {
                double s = 0.0;
                for (int k = 0; k < n; k++) s += I[c * n + k] * t2[a + m * (b + m * k)];
                qg[a + m * (b + m * c)] = s;
            }
}

/* Projection Gauss -> GLL with I^T (Algorithm 2, three 1D contractions):
 *   u1[c][b][i] = sum_a I[a][i] qg[c][b][a]
 *   u2[c][j][i] = sum_b I[b][j] u1[c][b][i]
 *   out[k][j][i] = sum_c I[c][k] u2[c][j][i]  */
static void project(int n, int m, const double *I, const double *qg, double *out,
                    double *u1, double *u2)
{
    for (int c = 0; c < m; c++)
        for (int b = 0; b < m; b++)
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int a = 0; a < m; a++) s += I[a * n + i] * qg[a + m * (b + m * c)];
                u1[i + n * (b + m * c)] = s;
            }
    for (int c = 0; c < m; c++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int b = 0; b < m; b++) s += I[b * n + j] * u1[i + n * (b + m * c)];
                u2[i + n * (j + n * c)] = s;
            }
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int c = 0; c < m; c++) s += I[c * n + k] * u2[i + n * (j + n * c)];
                out[i + n * (j + n * k)] = s;
            }
}

/* BP1.0 (Algorithm 3): Mq = I^T J I q per element. */
int or_bp1(int N, int64_t E, const double *wJ, const double *q, double *Mq)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1, m = N + 2;
    int64_t np = (int64_t)n * n * n, mp = (int64_t)m * m * m;
    double I[OR_MAXQ * OR_MAXQ];
    or_basis(N, NULL, NULL, NULL, NULL, I, NULL, NULL);
#pragma omp parallel
    {
        double *qg = malloc(sizeof(double) * mp);
        double *t1 = malloc(sizeof(double) * mp);
        double *t2 = malloc(sizeof(double) * mp);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < E; e++) {
            interpolate(n, m, I, q + e * np, qg, t1, t2);
            for (int64_t p = 0; p < mp; p++) qg[p] *= wJ[e * mp + p];
            project(n, m, I, qg, Mq + e * np, t1, t2);
        }
        free(qg);
        free(t1);
        free(t2);
    }
    return 0;
}

/* Stiffness-plus-mass kernel of Algorithm 4 on a q^3 grid with 1D
 * differentiation matrix Dm (q x q), geometric factors g (7 planes) and the
 * field u at the same points; result v (q^3):
 *   ur[k][j][i] = sum_n Dm[i][n] u[k][j][n]     (d/dr)
 *   us[k][j][i] = sum_n Dm[j][n] u[k][n][i]     (d/ds)
 *   ut[k][j][i] = sum_n Dm[k][n] u[n][j][i]     (d/dt)
 *   [Rr Rs Rt] = G [ur us ut]                   (chain rule, G symmetric)
 *   v[k][j][i] = lambda wJ u + sum_n Dm[n][i] Rr[k][j][n]
 *                + Dm[n][j] Rs[k][n][i] + Dm[n][k] Rt[n][j][i]  */
static void stiff_grid(int q, const double *Dm, const double *g, double lambda,
                       const double *u, double *v, double *Rr, double *Rs, double *Rt)
{
    int64_t P = (int64_t)q * q * q;
    for (int k = 0; k < q; k++)
        for (int j = 0; j < q; j++)
            for (int i = 0; i < q; i++) {
                double ur = 0.0, us = 0.0, ut = 0.0;
                for (int n = 0; n < q; n++) {
                    ur += Dm[i * q + n] * u[n + q * (j + q * k)];
                    us += Dm[j * q + n] * u[i + q * (n + q * k)];
                    ut += Dm[k * q + n] * u[i + q * (j + q * n)];
                }
                int64_t p = i + q * (j + q * k);
                double Grr = g[0 * P + p], Grs = g[1 * P + p], Grt = g[2 * P + p];
                double Gss = g[3 * P + p], Gst = g[4 * P + p], Gtt = g[5 * P + p];
                Rr[p] = Grr * ur + Grs * us + Grt * ut;
                Rs[p] = Grs * ur + Gss * us + Gst * ut;
                Rt[p] = Grt * ur + Gst * us + Gtt * ut;
            }
    for (int k = 0; k < q; k++)
        for (int j = 0; j < q; j++)
            for (int i = 0; i < q; i++) {
                int64_t p = i + q * (j + q * k);
                double s = lambda * g[6 * P + p] * u[p];
                for (int n = 0; n < q; n++) {
                    s += Dm[n * q + i] * Rr[n + q * (j + q * k)];
                    s += Dm[n * q + j] * Rs[i + q * (n + q * k)];
                    s += Dm[n * q + k] * Rt[i + q * (j + q * n)];
                }
                v[p] = s;
            }
}

/* BP3.5 (Algorithm 4): Aq = D^T G D q + lambda J q at the GLL nodes. */
int or_bp35(int N, int64_t E, const double *geo, double lambda, const double *q, double *Aq)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1;
    int64_t np = (int64_t)n * n * n;
    double D[OR_MAXQ * OR_MAXQ];
    or_basis(N, NULL, NULL, NULL, NULL, NULL, D, NULL);
#pragma omp parallel
    {
        double *Rr = malloc(sizeof(double) * np);
        double *Rs = malloc(sizeof(double) * np);
        double *Rt = malloc(sizeof(double) * np);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < E; e++)
            stiff_grid(n, D, geo + e * 7 * np, lambda, q + e * np, Aq + e * np, Rr, Rs, Rt);
        free(Rr);
        free(Rs);
        free(Rt);
    }
    return 0;
}

/* BP3.0 (Algorithm 5): Aq = I^T (Dt^T G Dt + lambda J) I q, the lambda J
 * term acting on the interpolated field at the Gauss points. */
int or_bp30(int N, int64_t E, const double *geo, double lambda, const double *q, double *Aq)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1, m = N + 2;
    int64_t np = (int64_t)n * n * n, mp = (int64_t)m * m * m;
    double I[OR_MAXQ * OR_MAXQ], Dt[OR_MAXQ * OR_MAXQ];
    or_basis(N, NULL, NULL, NULL, NULL, I, NULL, Dt);
#pragma omp parallel
    {
        double *qg = malloc(sizeof(double) * mp);
        double *vg = malloc(sizeof(double) * mp);
        double *t1 = malloc(sizeof(double) * mp);
        double *t2 = malloc(sizeof(double) * mp);
        double *t3 = malloc(sizeof(double) * mp);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < E; e++) {
            interpolate(n, m, I, q + e * np, qg, t1, t2);
            stiff_grid(m, Dt, geo + e * 7 * mp, lambda, qg, vg, t1, t2, t3);
            project(n, m, I, vg, Aq + e * np, t1, t2);
        }
        free(qg);
        free(vg);
        free(t1);
        free(t2);
        free(t3);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dense element matrices by brute force (no sum factorisation)       */
/* ------------------------------------------------------------------ */

/* The element matrix of one element, built entry by entry from the
 * quadrature sums of Section 4 (eq. massQuad, stiffQuad, stiffQuad2):
 *   A[p][p'] = sum_{quad pts} W (grad l_p')^T G (grad l_p) + lambda W |J| l_p' l_p
 * with grad taken in (r,s,t) and G = |J| X^{-1} X^{-T} evaluated at the point.
 * rule 0: Gauss rule with N+2 points (BP1.0 / BP3.0); rule 1: GLL rule with
 * N+1 points (BP3.5).  stiff = 0 gives the mass matrix alone (lambda ignored).
 * A is n^3 x n^3 row-major, row = test function p' (output index). */
int or_dense_element(int N, int rule, int stiff, double lambda, const double *v, double *A)
{
    if (N < 1 || N > 6) return -1;
    int n = N + 1, m = N + 2;
    int q = rule ? n : m;
    double gr[OR_MAXQ], gw[OR_MAXQ], qx[OR_MAXQ], qw[OR_MAXQ];
    or_gll(N, gr, gw);
    if (rule) {
        memcpy(qx, gr, sizeof(double) * n);
        memcpy(qw, gw, sizeof(double) * n);
    } else {
        or_gauss(m, qx, qw);
    }
    int np = n * n * n;
    /* l_i and l_i' at each 1D quadrature point */
    double L[OR_MAXQ][OR_MAXQ], dL[OR_MAXQ][OR_MAXQ];
    for (int a = 0; a < q; a++)
        for (int i = 0; i < n; i++) {
            L[a][i] = lagrange(n, gr, i, qx[a]);
            dL[a][i] = lagrange_d1(n, gr, i, qx[a]);
        }
    memset(A, 0, sizeof(double) * np * np);
    double *gx = malloc(sizeof(double) * np), *gy = malloc(sizeof(double) * np);
    double *gz = malloc(sizeof(double) * np), *val = malloc(sizeof(double) * np);
    for (int c = 0; c < q; c++)
        for (int b = 0; b < q; b++)
            for (int a = 0; a < q; a++) {
                double G[3][3];
                double det = metric_at(v, qx[a], qx[b], qx[c], G);
                double W = qw[a] * qw[b] * qw[c];
                for (int k = 0; k < n; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            int p = i + n * (j + n * k);
                            val[p] = L[a][i] * L[b][j] * L[c][k];
                            gx[p] = dL[a][i] * L[b][j] * L[c][k];
                            gy[p] = L[a][i] * dL[b][j] * L[c][k];
                            gz[p] = L[a][i] * L[b][j] * dL[c][k];
                        }
                for (int pr = 0; pr < np; pr++)
                    for (int pc = 0; pc < np; pc++) {
                        double s = 0.0;
                        if (stiff) {
                            double u0 = gx[pc], u1 = gy[pc], u2 = gz[pc];
                            double t0 = G[0][0] * u0 + G[0][1] * u1 + G[0][2] * u2;
                            double t1 = G[1][0] * u0 + G[1][1] * u1 + G[1][2] * u2;
                            double t2 = G[2][0] * u0 + G[2][1] * u1 + G[2][2] * u2;
                            s = gx[pr] * t0 + gy[pr] * t1 + gz[pr] * t2;
                            s += lambda * det * val[pr] * val[pc];
                        } else {
                            s = det * val[pr] * val[pc];
                        }
                        A[(int64_t)pr * np + pc] += W * s;
                    }
            }
    free(gx);
    free(gy);
    free(gz);
    free(val);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Jacobi-preconditioned conjugate gradients on the unassembled        */
/* BP3.5 screened-Poisson system (block diagonal, Section 4)           */
/* ------------------------------------------------------------------ */

/* Diagonal of the BP3.5 operator D^T G D + lambda J (Algorithm 4) in
 * closed form: entry (p,p) sums G_ab (D_a)_{node,p} (D_b)_{node,p} over the
 * quadrature nodes; the D_r, D_s, D_t factors touch one line each, so
 *   diag_ijk = sum_n (D_ni^2 Grr_njk + D_nj^2 Gss_ink + D_nk^2 Gtt_ijn)
 *            + 2 (D_ii D_jj Grs + D_ii D_kk Grt + D_jj D_kk Gst)_ijk
 *            + lambda wJ_ijk. */
int or_bp35_diag(int N, int64_t E, const double *geo, double lambda, double *diag)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1;
    int64_t np = (int64_t)n * n * n;
    double D[OR_MAXQ * OR_MAXQ];
    or_basis(N, NULL, NULL, NULL, NULL, NULL, D, NULL);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; e++) {
        const double *g = geo + e * 7 * np;
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int64_t p = i + n * (j + n * k);
                    double s = 0.0;
                    for (int m2 = 0; m2 < n; m2++) {
                        s += D[m2 * n + i] * D[m2 * n + i] * g[0 * np + m2 + n * (j + n * k)];
                        s += D[m2 * n + j] * D[m2 * n + j] * g[3 * np + i + n * (m2 + n * k)];
                        s += D[m2 * n + k] * D[m2 * n + k] * g[5 * np + i + n * (j + n * m2)];
                    }
                    double Dii = D[i * n + i], Djj = D[j * n + j], Dkk = D[k * n + k];
                    s += 2.0 * (Dii * Djj * g[1 * np + p] + Dii * Dkk * g[2 * np + p] +
                                Djj * Dkk * g[4 * np + p]);
                    s += lambda * g[6 * np + p];
                    diag[e * np + p] = s;
                }
    }
    return 0;
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned CG (Saad, Iterative Methods for Sparse Linear
 * Systems, 2nd ed., Algorithm 9.1, with M = diag(A)) for A x = b, A the
 * BP3.5 operator, starting from the x passed in.  Stops when
 * ||r||_2 <= tol ||b||_2 or after maxit iterations.  Returns the number of
 * iterations (>= 0), -1 on bad arguments, -2 on breakdown (p.Ap <= 0);
 * *relres receives ||r||_2 / ||b||_2 of the recursively updated residual. */
int or_pcg_bp35(int N, int64_t E, const double *geo, double lambda, const double *b, double *x,
                double tol, int maxit, double *relres)
{
    if (N < 1 || N > OR_MAXN || E < 1) return -1;
    int64_t len = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
    double *r = malloc(sizeof(double) * len), *z = malloc(sizeof(double) * len);
    double *p = malloc(sizeof(double) * len), *Ap = malloc(sizeof(double) * len);
    double *dg = malloc(sizeof(double) * len);
    int it = 0, status = 0;
    or_bp35_diag(N, E, geo, lambda, dg);
    or_bp35(N, E, geo, lambda, x, Ap);
    for (int64_t i = 0; i < len; i++) r[i] = b[i] - Ap[i];
    double bn = sqrt(dot(len, b, b));
    if (bn == 0.0) bn = 1.0;
    for (int64_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
    for (int64_t i = 0; i < len; i++) p[i] = z[i];
    double rz = dot(len, r, z);
    double rn = sqrt(dot(len, r, r));
    while (rn > tol * bn && it < maxit) {
        or_bp35(N, E, geo, lambda, p, Ap);
        double pAp = dot(len, p, Ap);
        if (!(pAp > 0.0)) {
            status = -2;
            break;
        }
        double alpha = rz / pAp;
        for (int64_t i = 0; i < len; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        for (int64_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
        double rz_new = dot(len, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < len; i++) p[i] = z[i] + beta * p[i];
        rn = sqrt(dot(len, r, r));
        it++;
    }
    if (relres) *relres = rn / bn;
    free(r);
    free(z);
    free(p);
    free(Ap);
    free(dg);
    return status ? status : it;
}

/* Diagonal of the BP3.0 operator I^T (Dt^T G Dt + lambda J) I (Algorithm 5)
 * entry by entry: with B = I (B_ai = l_i(rt_a)) and C = Dt I (C_ai =
 * l_i'(rt_a)) the gradient of basis function (i,j,k) at Gauss point (a,b,c)
 * is (C_ai B_bj B_ck, B_ai C_bj B_ck, B_ai B_bj C_ck), so
 *   diag_ijk = sum_abc [ g^T G g + lambda wJ (B_ai B_bj B_ck)^2 ]. */
int or_bp30_diag(int N, int64_t E, const double *geo, double lambda, double *diag)
{
    if (N < 1 || N > OR_MAXN) return -1;
    int n = N + 1, m = N + 2;
    int64_t np = (int64_t)n * n * n, mp = (int64_t)m * m * m;
    double I[OR_MAXQ * OR_MAXQ], Dt[OR_MAXQ * OR_MAXQ], Cm[OR_MAXQ * OR_MAXQ];
    or_basis(N, NULL, NULL, NULL, NULL, I, NULL, Dt);
    for (int a = 0; a < m; a++)
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int b = 0; b < m; b++) s += Dt[a * m + b] * I[b * n + i];
            Cm[a * n + i] = s;
        }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; e++) {
        const double *g = geo + e * 7 * mp;
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    double s = 0.0;
                    for (int c = 0; c < m; c++)
                        for (int b = 0; b < m; b++)
                            for (int a = 0; a < m; a++) {
                                int64_t p = a + m * (b + m * c);
                                double gr = Cm[a * n + i] * I[b * n + j] * I[c * n + k];
                                double gs = I[a * n + i] * Cm[b * n + j] * I[c * n + k];
                                double gt = I[a * n + i] * I[b * n + j] * Cm[c * n + k];
                                double v = I[a * n + i] * I[b * n + j] * I[c * n + k];
                                s += g[0 * mp + p] * gr * gr + g[3 * mp + p] * gs * gs + g[5 * mp + p] * gt * gt;
                                s += 2.0 * (g[1 * mp + p] * gr * gs + g[2 * mp + p] * gr * gt + g[4 * mp + p] * gs * gt);
                                s += lambda * g[6 * mp + p] * v * v;
                            }
                    diag[e * np + i + n * (j + n * k)] = s;
                }
    }
    return 0;
}

/* Jacobi-preconditioned CG for the BP3.0 system, as or_pcg_bp35. */
int or_pcg_bp30(int N, int64_t E, const double *geo, double lambda, const double *b, double *x,
                double tol, int maxit, double *relres)
{
    if (N < 1 || N > OR_MAXN || E < 1) return -1;
    int64_t len = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
    double *r = malloc(sizeof(double) * len), *z = malloc(sizeof(double) * len);
    double *p = malloc(sizeof(double) * len), *Ap = malloc(sizeof(double) * len);
    double *dg = malloc(sizeof(double) * len);
    int it = 0, status = 0;
    or_bp30_diag(N, E, geo, lambda, dg);
    or_bp30(N, E, geo, lambda, x, Ap);
    for (int64_t i = 0; i < len; i++) r[i] = b[i] - Ap[i];
    double bn = sqrt(dot(len, b, b));
    if (bn == 0.0) bn = 1.0;
    for (int64_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
    for (int64_t i = 0; i < len; i++) p[i] = z[i];
    double rz = dot(len, r, z);
    double rn = sqrt(dot(len, r, r));
    while (rn > tol * bn && it < maxit) {
        or_bp30(N, E, geo, lambda, p, Ap);
        double pAp = dot(len, p, Ap);
        if (!(pAp > 0.0)) {
            status = -2;
            break;
        }
        double alpha = rz / pAp;
        for (int64_t i = 0; i < len; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        for (int64_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
        double rz_new = dot(len, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < len; i++) p[i] = z[i] + beta * p[i];
        rn = sqrt(dot(len, r, r));
        it++;
    }
    if (relres) *relres = rn / bn;
    free(r);
    free(z);
    free(p);
    free(Ap);
    free(dg);
    return status ? status : it;
}
