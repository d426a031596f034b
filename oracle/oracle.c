/*
 * oracle.c -- plain, slow FP64 CPU reference for the discretised
 * Lippmann-Schwinger operator of Gujjula & Ambikasaran, "A new Directional
 * Algebraic Fast Multipole Method based iterative solver for the
 * Lippmann-Schwinger equation accelerated with HODLR preconditioner"
 * (arXiv 2204.00326).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code with the CUDA library.
 *
 * What it computes (all in double / double complex):
 *   - Chebyshev first-kind nodes of a p x p leaf grid (Section 2, Eq. 7-9);
 *   - the interpolation matrix Q (Eq. 9b) and its pseudo-inverse
 *     Q^+ = (Q^T Q)^{-1} Q^T written out from the definition (Eq. 10);
 *   - the Helmholtz Green's function G = (i/4) H0^(1)(kappa |x-y|) (Eq. 5-6)
 *     with H0^(1) = J0 + i Y0 taken from the C library's j0/y0;
 *   - the entries K_ij = int_{B(j)} G(x_i,y) L_{j'}(y) dy, where
 *     L_{j'} = sum_l Q^+_{l,j'} b_l is the least-squares cardinal function
 *     of Eq. 11, so that A = I + kappa^2 diag(q) K (Eq. 13);
 *   - rows of K, the matrix-vector product A v row by row, and a plain
 *     Gaussian-elimination LU solve of A psi = f (Eq. 12a);
 *   - the point N-body potential of Experiment 1 (Section 6.2) by direct
 *     summation over the same nodes;
 *   - the interpolant psi(x) (Eq. 7) and its volume potential at arbitrary
 *     points, the ingredients of the error function E(x) (Section 6.1).
 *
 * Quadrature (a reading: the paper names "adaptive Gauss quadrature" and
 * Boost's Hankel function, Section 2.3, but gives no rule): the reference
 * square of the source box is split at the target point, then cells are
 * bisected until each is at least half its diagonal away from the target,
 * where an m x m tensor Gauss-Legendre rule is used; cells that touch the
 * target and are smaller than a fixed size get a Duffy (collapsed triangle)
 * rule, which removes the logarithmic singularity of Y0.  Far boxes need a
 * single cell.  Accuracy is pinned by the tests against scipy's adaptive
 * quadrature, a manufactured solution and symmetry invariants.
 *
 * Ordering conventions (shared with the library as a convention only):
 *   leaf boxes in Morton (Z) order with the x bit below the y bit; inside a
 *   leaf, point i' = k1 + p*k2 with node zeta_k = -cos((2k+1) pi / (2p)).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_MAX_P 12
#define OR_MAX_M 64
#define OR_MAX_NP (OR_MAX_P * (OR_MAX_P + 1) / 2)

/* ------------------------------------------------------------------ */
/* 1-D building blocks                                                 */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1,1] by Newton's method on P_m. */
int or_gauss_legendre(int m, double* x, double* w)
{
    if (m < 1 || m > OR_MAX_M) return 1;
    for (int i = 0; i < m; i++) {
        double z = cos(M_PI * (i + 0.75) / (m + 0.5));
        double pm = 0.0, pm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p0 = 1.0; p1 = z; }
            pm = p1;
            pm1 = p0;
            dp = m * (z * pm - pm1) / (z * z - 1.0);
            double dz = pm / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p0 = 1.0; p1 = z; }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Chebyshev polynomial of the first kind T_n(x) by the three-term recurrence. */
double or_cheb_T(int n, double x)
{
    if (n == 0) return 1.0;
    double t0 = 1.0, t1 = x;
    for (int k = 2; k <= n; k++) {
        double t2 = 2.0 * x * t1 - t0;
        t0 = t1;
        t1 = t2;
    }
    return t1;
}

/* First-kind Chebyshev nodes on [-1,1] in ascending order (Section 2). */
void or_cheb_nodes(int p, double* z)
{
    for (int k = 0; k < p; k++) z[k] = -cos((2.0 * k + 1.0) * M_PI / (2.0 * p));
}

/* Number of 2-D polynomials of total degree < p: N_p = p(p+1)/2 (Section 2.2). */
int or_basis_count(int p) { return p * (p + 1) / 2; }

/* Basis b_l(e1,e2) = T_a(e1) T_b(e2), a+b < p, ordered by total degree then
 * by decreasing a. */
void or_basis_degrees(int p, int* a, int* b)
{
    int l = 0;
    for (int d = 0; d < p; d++)
        for (int aa = d; aa >= 0; aa--) {
            a[l] = aa;
            b[l] = d - aa;
            l++;
        }
}

/* ------------------------------------------------------------------ */
/* Interpolation matrix and pseudo-inverse (Eq. 9b, Eq. 10)            */
/* ------------------------------------------------------------------ */

/* Q (p^2 x Np, row-major): Q[i'][l] = b_l(zeta_{k1}, zeta_{k2}), i' = k1 + p k2. */
int or_qmatrix(int p, double* Q)
{
    if (p < 1 || p > OR_MAX_P) return 1;
    int np = or_basis_count(p);
    int a[OR_MAX_NP], b[OR_MAX_NP];
    double z[OR_MAX_P];
    or_basis_degrees(p, a, b);
    or_cheb_nodes(p, z);
    for (int k2 = 0; k2 < p; k2++)
        for (int k1 = 0; k1 < p; k1++)
            for (int l = 0; l < np; l++)
                Q[(k1 + p * k2) * np + l] = or_cheb_T(a[l], z[k1]) * or_cheb_T(b[l], z[k2]);
    return 0;
}

/* Solve M X = R (M: n x n, R: n x nr, both row-major, overwritten) by
 * Gaussian elimination with partial pivoting; X is left in R. */
static int gauss_solve_real(int n, double* M, int nr, double* R)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
        if (M[piv * n + c] == 0.0) return 4;
        if (piv != c) {
            for (int k = 0; k < n; k++) { double t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t; }
            for (int k = 0; k < nr; k++) { double t = R[c * nr + k]; R[c * nr + k] = R[piv * nr + k]; R[piv * nr + k] = t; }
        }
        for (int r = c + 1; r < n; r++) {
            double f = M[r * n + c] / M[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; k++) M[r * n + k] -= f * M[c * n + k];
            for (int k = 0; k < nr; k++) R[r * nr + k] -= f * R[c * nr + k];
        }
    }
    for (int c = n - 1; c >= 0; c--) {
        for (int k = 0; k < nr; k++) {
            double s = R[c * nr + k];
            for (int j = c + 1; j < n; j++) s -= M[c * n + j] * R[j * nr + k];
            R[c * nr + k] = s / M[c * n + c];
        }
    }
    return 0;
}

/* Q^+ (Np x p^2, row-major) = (Q^T Q)^{-1} Q^T, the pseudo-inverse of the
 * full-column-rank Q of Eq. 9b (Eq. 10). */
int or_qpinv(int p, double* Qp)
{
    if (p < 1 || p > OR_MAX_P) return 1;
    int np = or_basis_count(p), n2 = p * p;
    double* Q = malloc(sizeof(double) * n2 * np);
    double* M = malloc(sizeof(double) * np * np);
    or_qmatrix(p, Q);
    for (int r = 0; r < np; r++)
        for (int c = 0; c < np; c++) {
            double s = 0.0;
            for (int i = 0; i < n2; i++) s += Q[i * np + r] * Q[i * np + c];
            M[r * np + c] = s;
        }
    for (int r = 0; r < np; r++)
        for (int i = 0; i < n2; i++) Qp[r * n2 + i] = Q[i * np + r];
    int st = gauss_solve_real(np, M, n2, Qp);
    free(Q);
    free(M);
    return st;
}

/* ------------------------------------------------------------------ */
/* Green's function (Eq. 5-6)                                          */
/* ------------------------------------------------------------------ */

/* H0^(1)(z) = J0(z) + i Y0(z) for z > 0. */
void or_hankel0(double z, double* re, double* im)
{
    *re = j0(z);
    *im = y0(z);
}

/* G(r) = (i/4) H0^(1)(kappa r). */
static inline cplx green(double kappa, double r)
{
    double z = kappa * r;
    return 0.25 * I * (j0(z) + I * y0(z));
}

/* ------------------------------------------------------------------ */
/* Integrals of G times the basis over the reference square            */
/* ------------------------------------------------------------------ */

typedef struct {
    int p, np, m;
    int a[OR_MAX_NP], b[OR_MAX_NP];
    double gx[OR_MAX_M], gw[OR_MAX_M];
    double kb;       /* kappa * beta: wavenumber in reference coordinates */
    double tx, ty;   /* target in reference coordinates of the source box */
    double dmin;     /* size below which a corner cell gets the Duffy rule */
    cplx acc[OR_MAX_NP];
    int err;
} integ_ctx;

/* Accumulate w * G(|t - eta|) * b_l(eta) for all l. */
static void add_point(integ_ctx* c, double ex, double ey, double w)
{
    double dx = ex - c->tx, dy = ey - c->ty;
    double r = sqrt(dx * dx + dy * dy);
    cplx g = green(c->kb, r) * w;
    double Ta[OR_MAX_P], Tb[OR_MAX_P];
    Ta[0] = 1.0; Tb[0] = 1.0;
    if (c->p > 1) { Ta[1] = ex; Tb[1] = ey; }
    for (int k = 2; k < c->p; k++) {
        Ta[k] = 2.0 * ex * Ta[k - 1] - Ta[k - 2];
        Tb[k] = 2.0 * ey * Tb[k - 1] - Tb[k - 2];
    }
    for (int l = 0; l < c->np; l++) c->acc[l] += g * (Ta[c->a[l]] * Tb[c->b[l]]);
}

/* m x m tensor Gauss-Legendre rule on [x0,x1] x [y0,y1]. */
static void rule_tensor(integ_ctx* c, double x0, double x1, double y0, double y1)
{
    double hx = 0.5 * (x1 - x0), cx = 0.5 * (x1 + x0);
    double hy = 0.5 * (y1 - y0), cy = 0.5 * (y1 + y0);
    for (int i = 0; i < c->m; i++)
        for (int j = 0; j < c->m; j++)
            add_point(c, cx + hx * c->gx[i], cy + hy * c->gx[j], hx * hy * c->gw[i] * c->gw[j]);
}

/* Duffy rule on the triangle (t, P0, P1): y = t + u ((1-s) P0 + s P1 - t),
 * u, s in [0,1], Jacobian u |det(P0 - t, P1 - t)|. */
static void rule_duffy_triangle(integ_ctx* c, double p0x, double p0y, double p1x, double p1y)
{
    double ax = p0x - c->tx, ay = p0y - c->ty, bx = p1x - c->tx, by = p1y - c->ty;
    double det = fabs(ax * by - ay * bx);
    for (int i = 0; i < c->m; i++) {
        double u = 0.5 * (c->gx[i] + 1.0), wu = 0.5 * c->gw[i];
        for (int j = 0; j < c->m; j++) {
            double s = 0.5 * (c->gx[j] + 1.0), ws = 0.5 * c->gw[j];
            double ex = c->tx + u * ((1.0 - s) * ax + s * bx);
            double ey = c->ty + u * ((1.0 - s) * ay + s * by);
            add_point(c, ex, ey, wu * ws * u * det);
        }
    }
}

static double dist_point_rect(double tx, double ty, double x0, double x1, double y0, double y1)
{
    double dx = (tx < x0) ? x0 - tx : (tx > x1 ? tx - x1 : 0.0);
    double dy = (ty < y0) ? y0 - ty : (ty > y1 ? ty - y1 : 0.0);
    return sqrt(dx * dx + dy * dy);
}

static void integrate_cell(integ_ctx* c, double x0, double x1, double y0, double y1, int depth)
{
    double d = dist_point_rect(c->tx, c->ty, x0, x1, y0, y1);
    double D = hypot(x1 - x0, y1 - y0);
    if (d >= 0.5 * D) { rule_tensor(c, x0, x1, y0, y1); return; }
    int corner = (c->tx == x0 || c->tx == x1) && (c->ty == y0 || c->ty == y1);
    if (corner && D < c->dmin) {
        /* the two triangles with apex t that tile the cell */
        double ox = (c->tx == x0) ? x1 : x0, oy = (c->ty == y0) ? y1 : y0;
        rule_duffy_triangle(c, ox, c->ty, ox, oy);
        rule_duffy_triangle(c, ox, oy, c->tx, oy);
        return;
    }
    if (depth > 60) { c->err = 1; rule_tensor(c, x0, x1, y0, y1); return; }
    double wx = x1 - x0, wy = y1 - y0;
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
    if (wx > 2.0 * wy) {
        integrate_cell(c, x0, xm, y0, y1, depth + 1);
        integrate_cell(c, xm, x1, y0, y1, depth + 1);
    } else if (wy > 2.0 * wx) {
        integrate_cell(c, x0, x1, y0, ym, depth + 1);
        integrate_cell(c, x0, x1, ym, y1, depth + 1);
    } else {
        integrate_cell(c, x0, xm, y0, ym, depth + 1);
        integrate_cell(c, xm, x1, y0, ym, depth + 1);
        integrate_cell(c, x0, xm, ym, y1, depth + 1);
        integrate_cell(c, xm, x1, ym, y1, depth + 1);
    }
}

/*
 * I_l = int_{[-1,1]^2} (i/4) H0^(1)(kb |t - eta|) b_l(eta) d eta, l = 0..Np-1,
 * for a target t = (tx, ty) given in the reference coordinates of the source
 * box (Section 2.3).  The square is first cut at the target's coordinates so
 * that the singular point lies on cell corners only.  m is the Gauss-Legendre
 * order per cell, dmin the corner-cell size handled by the Duffy rule.
 * Output as interleaved (re, im) pairs.  Returns 0 on success.
 */
int or_basis_integrals(int p, double kb, double tx, double ty, int m, double dmin, double* out)
{
    if (p < 1 || p > OR_MAX_P || m < 1 || m > OR_MAX_M) return 1;
    integ_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = p;
    c.np = or_basis_count(p);
    c.m = m;
    or_basis_degrees(p, c.a, c.b);
    or_gauss_legendre(m, c.gx, c.gw);
    c.kb = kb;
    c.tx = tx;
    c.ty = ty;
    c.dmin = dmin;
    double xs[3] = {-1.0, 0, 1.0}, ys[3] = {-1.0, 0, 1.0};
    int nx = 2, ny = 2;
    if (tx > -1.0 && tx < 1.0) { xs[1] = tx; xs[2] = 1.0; nx = 3; } else { xs[1] = 1.0; }
    if (ty > -1.0 && ty < 1.0) { ys[1] = ty; ys[2] = 1.0; ny = 3; } else { ys[1] = 1.0; }
    for (int i = 0; i + 1 < nx; i++)
        for (int j = 0; j + 1 < ny; j++) integrate_cell(&c, xs[i], xs[i + 1], ys[j], ys[j + 1], 0);
    for (int l = 0; l < c.np; l++) {
        out[2 * l] = creal(c.acc[l]);
        out[2 * l + 1] = cimag(c.acc[l]);
    }
    return c.err ? 4 : 0;
}

/* ------------------------------------------------------------------ */
/* Grid, ordering and rows of K (Eq. 13)                               */
/* ------------------------------------------------------------------ */

/* Leaf (bx, by) from its Morton index: bit 2k -> x bit k, bit 2k+1 -> y bit k. */
static void morton_decode(long m, long* bx, long* by)
{
    long x = 0, y = 0;
    for (int k = 0; k < 31; k++) {
        x |= ((m >> (2 * k)) & 1L) << k;
        y |= ((m >> (2 * k + 1)) & 1L) << k;
    }
    *bx = x;
    *by = y;
}

typedef struct {
    int p, n2, np;
    long nb, N;
    double x0, x1, beta, kappa;
    double z[OR_MAX_P];
    double* Qp; /* Np x p^2 */
    int m;
    double dmin;
} grid_ctx;

static int grid_init(grid_ctx* g, int n_side, double x0, double x1, int p, double kappa)
{
    if (p < 1 || p > OR_MAX_P || n_side < p || n_side % p) return 1;
    g->p = p;
    g->n2 = p * p;
    g->np = or_basis_count(p);
    g->nb = n_side / p;
    long nb = g->nb;
    if (nb & (nb - 1)) return 1; /* leaves per side must be a power of two */
    g->N = (long)n_side * n_side;
    g->x0 = x0;
    g->x1 = x1;
    g->beta = (x1 - x0) / (2.0 * nb);
    g->kappa = kappa;
    or_cheb_nodes(p, g->z);
    g->Qp = malloc(sizeof(double) * g->np * g->n2);
    g->m = 20;
    g->dmin = 2e-6;
    return or_qpinv(p, g->Qp);
}

static void leaf_center(const grid_ctx* g, long leaf, double* ax, double* ay)
{
    long bx, by;
    morton_decode(leaf, &bx, &by);
    *ax = g->x0 + (2.0 * bx + 1.0) * g->beta;
    *ay = g->x0 + (2.0 * by + 1.0) * g->beta;
}

static void point_xy(const grid_ctx* g, long i, double* x, double* y)
{
    long leaf = i / g->n2;
    int ip = (int)(i % g->n2);
    double ax, ay;
    leaf_center(g, leaf, &ax, &ay);
    *x = ax + g->beta * g->z[ip % g->p];
    *y = ay + g->beta * g->z[ip / g->p];
}

/* Coordinates of all N unknowns in the library's ordering (xy: N x 2). */
int or_grid_nodes(int n_side, double x0, double x1, int p, double* xy)
{
    grid_ctx g;
    int st = grid_init(&g, n_side, x0, x1, p, 1.0);
    if (st) { free(g.Qp); return st; }
    for (long i = 0; i < g.N; i++) point_xy(&g, i, &xy[2 * i], &xy[2 * i + 1]);
    free(g.Qp);
    return 0;
}

/* Entries K(x, j) for one target point x against all p^2 sources of one leaf:
 * K = beta^2 sum_l Q^+_{l,j'} I_l  (Eq. 13 without the kappa^2 q factor). */
static int leaf_entries(const grid_ctx* g, double x, double y, long leaf, cplx* out)
{
    double ax, ay;
    leaf_center(g, leaf, &ax, &ay);
    double il[2 * OR_MAX_NP];
    int st = or_basis_integrals(g->p, g->kappa * g->beta, (x - ax) / g->beta, (y - ay) / g->beta, g->m, g->dmin, il);
    double b2 = g->beta * g->beta;
    for (int jp = 0; jp < g->n2; jp++) {
        cplx s = 0.0;
        for (int l = 0; l < g->np; l++) s += g->Qp[l * g->n2 + jp] * (il[2 * l] + I * il[2 * l + 1]);
        out[jp] = b2 * s;
    }
    return st;
}

/*
 * Rows of K (N columns each, complex interleaved, row-major) for the listed
 * row indices.  Parallel over rows when compiled with OpenMP.
 */
int or_K_rows(int n_side, double x0, double x1, int p, double kappa, long nrows, const long* rows, double* Kout)
{
    grid_ctx g;
    int st = grid_init(&g, n_side, x0, x1, p, kappa);
    if (st) { free(g.Qp); return st; }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (long r = 0; r < nrows; r++) {
        double x, y;
        point_xy(&g, rows[r], &x, &y);
        cplx blk[OR_MAX_P * OR_MAX_P];
        for (long leaf = 0; leaf < g.nb * g.nb; leaf++) {
            err |= leaf_entries(&g, x, y, leaf, blk);
            for (int jp = 0; jp < g.n2; jp++) {
                long j = leaf * g.n2 + jp;
                Kout[2 * (r * g.N + j)] = creal(blk[jp]);
                Kout[2 * (r * g.N + j) + 1] = cimag(blk[jp]);
            }
        }
    }
    free(g.Qp);
    return err;
}

/*
 * (A v)_i = v_i + kappa^2 q_i sum_j K_ij v_j for the listed rows, with the
 * entries of each row generated on the fly (Eq. 12a-13).  v, out complex
 * interleaved; q real (length N).  nrhs right-hand sides stored [N][nrhs].
 */
int or_matvec_rows(int n_side, double x0, double x1, int p, double kappa, const double* q, int nrhs,
                   const double* v, long nrows, const long* rows, double* out)
{
    grid_ctx g;
    int st = grid_init(&g, n_side, x0, x1, p, kappa);
    if (st) { free(g.Qp); return st; }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (long r = 0; r < nrows; r++) {
        long i = rows[r];
        double x, y;
        point_xy(&g, i, &x, &y);
        cplx blk[OR_MAX_P * OR_MAX_P];
        cplx acc[64];
        int nr = nrhs > 64 ? 64 : nrhs;
        for (int k = 0; k < nr; k++) acc[k] = 0.0;
        for (long leaf = 0; leaf < g.nb * g.nb; leaf++) {
            err |= leaf_entries(&g, x, y, leaf, blk);
            for (int jp = 0; jp < g.n2; jp++) {
                long j = leaf * g.n2 + jp;
                for (int k = 0; k < nr; k++) {
                    cplx vj = v[2 * (j * nrhs + k)] + I * v[2 * (j * nrhs + k) + 1];
                    acc[k] += blk[jp] * vj;
                }
            }
        }
        for (int k = 0; k < nr; k++) {
            cplx vi = v[2 * (i * nrhs + k)] + I * v[2 * (i * nrhs + k) + 1];
            cplx o = vi + kappa * kappa * q[i] * acc[k];
            out[2 * (r * nrhs + k)] = creal(o);
            out[2 * (r * nrhs + k) + 1] = cimag(o);
        }
    }
    free(g.Qp);
    return err;
}

/*
 * Fields of a grid solution psi_vec at m arbitrary points x (Section 6.1's
 * error function E(x)): psi(x) = sum_l Q^+(l,:) psi_vec^B b_l((x - alpha^B) /
 * beta) on the leaf B containing x (Eq. 7; zero outside the domain), and the
 * volume potential u(x) = sum_B sum_j' K(x, B, j') psi_vec^B_j' with the
 * entries of Eq. 13 at the off-grid target x (the same quadrature as the
 * rows of K).  psi complex interleaved (N), pts m x 2, u and psi_at m
 * complex interleaved.
 */
int or_field_eval(int n_side, double x0, double x1, int p, double kappa, const double* psi, long m, const double* pts, double* u,
                  double* psi_at)
{
    grid_ctx g;
    int st = grid_init(&g, n_side, x0, x1, p, kappa);
    if (st) { free(g.Qp); return st; }
    int a[OR_MAX_NP], b[OR_MAX_NP];
    or_basis_degrees(p, a, b);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (long k = 0; k < m; k++) {
        const double x = pts[2 * k], y = pts[2 * k + 1];
        cplx blk[OR_MAX_P * OR_MAX_P];
        cplx acc = 0.0;
        for (long leaf = 0; leaf < g.nb * g.nb; leaf++) {
            err |= leaf_entries(&g, x, y, leaf, blk);
            for (int jp = 0; jp < g.n2; jp++) {
                long j = leaf * g.n2 + jp;
                acc += blk[jp] * (psi[2 * j] + I * psi[2 * j + 1]);
            }
        }
        u[2 * k] = creal(acc);
        u[2 * k + 1] = cimag(acc);
        cplx pv = 0.0;
        double ex = (x - x0) / (2.0 * g.beta), ey = (y - x0) / (2.0 * g.beta);
        if (ex >= 0.0 && ey >= 0.0 && ex <= g.nb && ey <= g.nb) {
            long bx = (long)floor(ex), by = (long)floor(ey);
            if (bx > g.nb - 1) bx = g.nb - 1;
            if (by > g.nb - 1) by = g.nb - 1;
            long leaf = 0;
            for (int q = 0; q < 31; q++) leaf |= (((bx >> q) & 1L) << (2 * q)) | (((by >> q) & 1L) << (2 * q + 1));
            double tx = (x - (x0 + (2.0 * bx + 1.0) * g.beta)) / g.beta, ty = (y - (x0 + (2.0 * by + 1.0) * g.beta)) / g.beta;
            for (int l = 0; l < g.np; l++) {
                cplx cl = 0.0;
                for (int jp = 0; jp < g.n2; jp++) {
                    long j = leaf * g.n2 + jp;
                    cl += g.Qp[l * g.n2 + jp] * (psi[2 * j] + I * psi[2 * j + 1]);
                }
                pv += cl * or_cheb_T(a[l], tx) * or_cheb_T(b[l], ty);
            }
        }
        if (psi_at) {
            psi_at[2 * k] = creal(pv);
            psi_at[2 * k + 1] = cimag(pv);
        }
    }
    free(g.Qp);
    return err;
}

/*
 * Experiment 1's N-body potential (Section 6.2): charges v_j at the grid
 * nodes p_j, u_i = sum_{j != i} G(p_i, p_j) v_j with G = (i/4) H0^(1)(kappa
 * |p_i - p_j|), by direct summation for the listed rows (the paper's sum
 * runs over every j; the j = i term is singular and left out, a reading).
 * v, out complex interleaved, [N][nrhs].
 */
int or_nbody_rows(int n_side, double x0, double x1, int p, double kappa, int nrhs, const double* v, long nrows, const long* rows,
                  double* out)
{
    grid_ctx g;
    int st = grid_init(&g, n_side, x0, x1, p, kappa);
    if (st) { free(g.Qp); return st; }
    const long N = (long)n_side * n_side;
    double* xy = (double*)malloc(sizeof(double) * 2 * N);
    if (!xy) { free(g.Qp); return 2; }
    for (long j = 0; j < N; j++) point_xy(&g, j, &xy[2 * j], &xy[2 * j + 1]);
    int nr = nrhs > 64 ? 64 : nrhs;
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < nrows; r++) {
        long i = rows[r];
        cplx acc[64];
        for (int k = 0; k < nr; k++) acc[k] = 0.0;
        for (long j = 0; j < N; j++) {
            if (j == i) continue;
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            cplx gij = green(kappa, sqrt(dx * dx + dy * dy));
            for (int k = 0; k < nr; k++) acc[k] += gij * (v[2 * (j * nrhs + k)] + I * v[2 * (j * nrhs + k) + 1]);
        }
        for (int k = 0; k < nr; k++) {
            out[2 * (r * nrhs + k)] = creal(acc[k]);
            out[2 * (r * nrhs + k) + 1] = cimag(acc[k]);
        }
    }
    free(xy);
    free(g.Qp);
    return 0;
}

/*
 * Solve A x = b for a dense complex n x n matrix (row-major, interleaved,
 * overwritten by its LU factors) by Gaussian elimination with partial
 * pivoting.  b (n x nrhs, interleaved) is overwritten by x.
 */
int or_lu_solve(long n, double* A_, int nrhs, double* b_)
{
    cplx* A = (cplx*)A_;
    cplx* b = (cplx*)b_;
    for (long c = 0; c < n; c++) {
        long piv = c;
        double best = cabs(A[c * n + c]);
        for (long r = c + 1; r < n; r++) {
            double v = cabs(A[r * n + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return 4;
        if (piv != c) {
            for (long k = 0; k < n; k++) { cplx t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            for (int k = 0; k < nrhs; k++) { cplx t = b[c * nrhs + k]; b[c * nrhs + k] = b[piv * nrhs + k]; b[piv * nrhs + k] = t; }
        }
        cplx inv = 1.0 / A[c * n + c];
#pragma omp parallel for schedule(static)
        for (long r = c + 1; r < n; r++) {
            cplx f = A[r * n + c] * inv;
            if (f == 0.0) continue;
            A[r * n + c] = f;
            for (long k = c + 1; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            for (int k = 0; k < nrhs; k++) b[r * nrhs + k] -= f * b[c * nrhs + k];
        }
    }
    for (long c = n - 1; c >= 0; c--) {
        for (int k = 0; k < nrhs; k++) {
            cplx s = b[c * nrhs + k];
            for (long j = c + 1; j < n; j++) s -= A[c * n + j] * b[j * nrhs + k];
            b[c * nrhs + k] = s / A[c * n + c];
        }
    }
    return 0;
}

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
