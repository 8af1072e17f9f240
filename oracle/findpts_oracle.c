/*
 * findpts_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, brute-force FP64 CPU reference for the point-location
 * (findpts) and interpolation (findpts_eval) step of Schwarz-SEM overset
 * coupling (Mittal, Dutta, Fischer, arXiv 1811.04891, Sec. 2.1).  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 2.1): for a query point x* tagged with session j
 * (or untagged, j = -1), every element e with sub(e) != j is examined; x* is
 * inside e when some r in [-1,1]^3 satisfies x^e(r) = x*, where
 *     x^e(r,s,t) = sum_ijk x^e_ijk h_i(r) h_j(s) h_k(t)          (Sec. 1, 2)
 * is the isoparametric map on the GLL nodes.  r is found by a box-constrained
 * trust-region Newton minimisation of ||x^e(r) - x*||^2 started from the
 * closest mapped GLL node of e (Sec. 2.1).  Among subdomains that contain x*
 * the owner maximises the distance function delta^k(x*) (Sec. 2.1, Fig. 4).
 * The result is a code (inside / border / not found), subdomain, element and
 * (r,s,t); findpts_eval then returns sum_ijk f_ijk h_i h_j h_k at that point.
 *
 * The 2D variant (quadrilateral meshes, coords [2][E][n^2], r in [-1,1]^2;
 * the paper's 2D overset examples, Sec. 3) runs the same steps with the
 * double sum x^e(r,s) = sum_ij x^e_ij h_i(r) h_j(s): or_find_d / or_eval_d /
 * or_map_d with d = 2, or_dist_default_2d.
 *
 * Deliberately naive: the map and its Jacobian are full triple sums (no sum
 * factorisation), the Lagrange basis is the product formula, every element is
 * a candidate (a permissive prefilter is optional; a CPU test checks that it
 * never changes a result against the same search without it).
 *
 * Readings where the paper is silent (stated once, used everywhere):
 *  - INSIDE:  ||x^e(r) - x*||_2 <= tol_accept * h_e, h_e = diagonal of the
 *             box spanned by the element's nodes.
 *  - element tie (point on a shared face): lowest global element id.
 *  - owner tie: |delta_a - delta_b| <= tie_band * L (L = diagonal of the box
 *             spanned by all nodes) goes to the lower subdomain id.
 *  - BORDER:  no INSIDE element, smallest constrained residual d_min <=
 *             tol_border * h_e; element = lowest id with residual <=
 *             d_min + tie_band * L.
 *  - NOT_FOUND: elem = sub = -1, r = 0, dist2 = +inf; eval gives NaN.
 *  - non-finite query coordinates: NOT_FOUND.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMAX 16          /* at most 16 GLL points per direction (N <= 15) */
#define OR_INSIDE 0
#define OR_BORDER 1
#define OR_NOT_FOUND 2

/* ------------------------------------------------------------------------ */
/* GLL nodes and weights                                                    */
/* ------------------------------------------------------------------------ */

/* Legendre P_N(x) and P_{N-1}(x) by the three-term recurrence
   (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_pair(int N, double x, double *pN, double *pNm1)
{
    double p0 = 1.0, p1 = x;
    if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
    for (int k = 1; k < N; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pN = p1;
    *pNm1 = p0;
}

/* GLL points of order N: -1, the N-1 roots of P_N', +1 (Sec. 2: nodal bases
   on the Gauss-Lobatto-Legendre points).  Interior roots by Newton on P_N',
   with P_N' = N (x P_N - P_{N-1}) / (x^2 - 1) and P_N'' from Legendre's
   equation (1-x^2) P'' - 2x P' + N(N+1) P = 0.  Weights (GLL quadrature)
   w_i = 2 / (N (N+1) P_N(x_i)^2).  Returns 0 on success. */
int or_gll(int N, double *x, double *w)
{
    if (N < 1 || N >= OR_NMAX) return -1;
    x[0] = -1.0;
    x[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double z = -cos(M_PI * (double)i / (double)N);   /* Chebyshev-GL guess */
        for (int it = 0; it < 100; ++it) {
            double p, q;
            legendre_pair(N, z, &p, &q);
            double dp = N * (z * p - q) / (z * z - 1.0);
            double d2p = (2.0 * z * dp - N * (N + 1.0) * p) / (1.0 - z * z);
            double dz = dp / d2p;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        x[i] = z;
    }
    for (int i = 0; i <= N / 2; ++i) {          /* exact antisymmetry */
        double a = 0.5 * (x[N - i] - x[i]);
        x[i] = -a;
        x[N - i] = a;
    }
    if (N % 2 == 0) x[N / 2] = 0.0;
    if (w) {
        for (int i = 0; i <= N; ++i) {
            double p, q;
            legendre_pair(N, x[i], &p, &q);
            w[i] = 2.0 / (N * (N + 1.0) * p * p);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lagrange basis on the GLL points: product formula and its derivative     */
/* ------------------------------------------------------------------------ */

/* h_i(r) = prod_{m != i} (r - x_m) / (x_i - x_m);
   h_i'(r) = sum_{k != i} 1/(x_i - x_k) prod_{m != i,k} (r - x_m)/(x_i - x_m). */
void or_lagrange(int N, const double *xg, double r, double *h, double *dh)
{
    for (int i = 0; i <= N; ++i) {
        double p = 1.0;
        for (int m = 0; m <= N; ++m)
            if (m != i) p *= (r - xg[m]) / (xg[i] - xg[m]);
        h[i] = p;
        if (dh) {
            double s = 0.0;
            for (int k = 0; k <= N; ++k) {
                if (k == i) continue;
                double q = 1.0 / (xg[i] - xg[k]);
                for (int m = 0; m <= N; ++m)
                    if (m != i && m != k) q *= (r - xg[m]) / (xg[i] - xg[m]);
                s += q;
            }
            dh[i] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Isoparametric map and Jacobian: full triple sum                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, n;
    int d;                       /* dimension: 3 (hexahedra) or 2 (quadrilaterals) */
    const double *xg;            /* GLL points */
    const double *X[3];          /* this element's node coordinates, n^d each (X[2] unused in 2D) */
} or_elem;

/* x(r) = sum_ijk X_ijk h_i(r0) h_j(r1) h_k(r2) and J[a][b] = dx_a/dr_b
   (J stored with row stride 3).  In 2D: x(r) = sum_ij X_ij h_i(r0) h_j(r1). */
static void or_map_elem(const or_elem *el, const double r[3], double x[3], double J[9])
{
    int n = el->n, N = el->N;
    double h[3][OR_NMAX], dh[3][OR_NMAX];
    if (el->d == 2) {
        for (int d = 0; d < 2; ++d) or_lagrange(N, el->xg, r[d], h[d], dh[d]);
        for (int a = 0; a < 2; ++a) {
            double v = 0.0, vr = 0.0, vs = 0.0;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double c = el->X[a][i + n * j];
                    v  += c * h[0][i]  * h[1][j];
                    vr += c * dh[0][i] * h[1][j];
                    vs += c * h[0][i]  * dh[1][j];
                }
            x[a] = v;
            if (J) { J[3 * a + 0] = vr; J[3 * a + 1] = vs; }
        }
        return;
    }
    for (int d = 0; d < 3; ++d) or_lagrange(N, el->xg, r[d], h[d], dh[d]);
    for (int a = 0; a < 3; ++a) {
        double v = 0.0, vr = 0.0, vs = 0.0, vt = 0.0;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double c = el->X[a][i + n * (j + n * k)];
                    v  += c * h[0][i]  * h[1][j]  * h[2][k];
                    vr += c * dh[0][i] * h[1][j]  * h[2][k];
                    vs += c * h[0][i]  * dh[1][j] * h[2][k];
                    vt += c * h[0][i]  * h[1][j]  * dh[2][k];
                }
        x[a] = v;
        if (J) { J[3 * a + 0] = vr; J[3 * a + 1] = vs; J[3 * a + 2] = vt; }
    }
}

/* Exported for tests: map M points (r given [d][M]) through element e of a
   d-dimensional mesh (coords [d][E][n^d]); x [d][M], J [d*d][M] row-major. */
void or_map_d(int d, int N, const double *coords, int64_t E, int64_t e, int64_t M,
              const double *r, double *x, double *J)
{
    double xg[OR_NMAX];
    or_gll(N, xg, NULL);
    int n = N + 1, nd = d == 2 ? n * n : n * n * n;
    or_elem el = { N, n, d, xg, { coords + e * nd, coords + (E + e) * nd, d == 3 ? coords + (2 * E + e) * nd : NULL } };
    for (int64_t m = 0; m < M; ++m) {
        double rr[3] = { r[m], r[M + m], d == 3 ? r[2 * M + m] : 0.0 }, xx[3], JJ[9];
        or_map_elem(&el, rr, xx, JJ);
        for (int a = 0; a < d; ++a) x[a * M + m] = xx[a];
        if (J)
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) J[(a * d + b) * M + m] = JJ[3 * a + b];
    }
}

void or_map(int N, const double *coords, int64_t E, int64_t e, int64_t M,
            const double *r, double *x, double *J)
{
    or_map_d(3, N, coords, E, e, M, r, x, J);
}

/* ------------------------------------------------------------------------ */
/* Box-constrained trust-region Newton on phi(r) = 1/2 ||x(r) - x*||^2       */
/* (Sec. 2.1: trust-region Newton minimising ||x^e(r) - x*||^2)              */
/* ------------------------------------------------------------------------ */

/* Solve the k x k symmetric positive (semi)definite system A z = b by
   Gaussian elimination with partial pivoting; returns 0 if singular. */
static int solve_small(int k, double A[3][3], double b[3], double z[3])
{
    int p[3] = { 0, 1, 2 };
    double M[3][4];
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) M[i][j] = A[i][j];
        M[i][3] = b[i];
    }
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (fabs(M[i][c]) > fabs(M[piv][c])) piv = i;
        if (M[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int j = 0; j < 4; ++j) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
        for (int i = c + 1; i < k; ++i) {
            double f = M[i][c] / M[c][c];
            for (int j = c; j < 4; ++j) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        double s = M[i][3];
        for (int j = i + 1; j < k; ++j) s -= M[i][j] * z[j];
        z[i] = s / M[i][i];
    }
    (void)p;
    return 1;
}

/* Newton from r (in/out).  Returns the final residual norm ||x(r) - x*||.
   Each iteration: residual f = x(r) - x*, gradient g = J^T f.  A coordinate
   sitting on a bound whose gradient component pushes it outward is frozen
   (active set); on the free coordinates the Gauss-Newton step solves
   (J_F^T J_F) d_F = -J_F^T f (the plain Newton step J d = -f when all three
   are free).  The step is limited to the trust radius (infinity norm), then
   shortened along its direction so that it stays in the box.  It is accepted
   when the actual decrease of phi is positive; the radius doubles when the
   actual/predicted ratio exceeds 0.75 and shrinks to a quarter of the step
   length when it is below 0.25 (standard trust-region updates).  Stop when an
   accepted step is below 1e-13 in every coordinate, the residual is exactly
   zero, the radius collapses below 1e-15, or after max_it iterations. */
static double sumsq(int d, const double *v)
{
    double s = v[0] * v[0];
    for (int a = 1; a < d; ++a) s += v[a] * v[a];
    return s;
}

static double or_newton(const or_elem *el, const double xs[3], double r[3], int max_it)
{
    const int dim = el->d;
    double x[3], J[9], f[3] = { 0, 0, 0 };
    or_map_elem(el, r, x, J);
    for (int a = 0; a < dim; ++a) f[a] = x[a] - xs[a];
    double phi = 0.5 * sumsq(dim, f);
    double rho = 1.0;
    for (int it = 0; it < max_it; ++it) {
        if (phi == 0.0) break;
        double g[3] = { 0, 0, 0 };
        for (int b = 0; b < dim; ++b) {
            g[b] = J[b] * f[0];
            for (int a = 1; a < dim; ++a) g[b] += J[3 * a + b] * f[a];
        }
        /* active set: bound coordinates whose descent direction points out
           of the box; grown while the Gauss-Newton step on the free
           coordinates would push a free bound coordinate outward */
        int act[3] = { 1, 1, 1 };
        for (int b = 0; b < dim; ++b)
            act[b] = (r[b] <= -1.0 && g[b] > 0.0) || (r[b] >= 1.0 && g[b] < 0.0);
        double d[3];
        int k;
        for (int pass = 0; pass < 4; ++pass) {
            int fr[3];
            k = 0;
            for (int b = 0; b < dim; ++b) if (!act[b]) fr[k++] = b;
            d[0] = d[1] = d[2] = 0.0;
            if (k == 0) break;
            double A[3][3], rhs[3], z[3];
            for (int p = 0; p < k; ++p) {
                for (int q = 0; q < k; ++q) {
                    double sacc = 0.0;
                    for (int a = 0; a < dim; ++a) sacc += J[3 * a + fr[p]] * J[3 * a + fr[q]];
                    A[p][q] = sacc;
                }
                rhs[p] = -g[fr[p]];
            }
            if (!solve_small(k, A, rhs, z))
                for (int p = 0; p < k; ++p) z[p] = rhs[p];   /* singular: steepest descent */
            for (int p = 0; p < k; ++p) d[fr[p]] = z[p];
            int grew = 0;
            for (int b = 0; b < dim; ++b)
                if (!act[b] && ((r[b] <= -1.0 && d[b] < 0.0) || (r[b] >= 1.0 && d[b] > 0.0))) {
                    act[b] = 1;
                    grew = 1;
                }
            if (!grew) break;
        }
        if (k == 0) break;                        /* KKT point at a vertex */
        /* trust region (infinity norm) */
        double dn = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
        if (dn == 0.0) break;
        if (dn > rho) for (int b = 0; b < 3; ++b) d[b] *= rho / dn;
        /* stay in the box: largest t <= 1 with r + t d in [-1,1]^3 */
        double t = 1.0;
        for (int b = 0; b < dim; ++b) {
            if (d[b] > 0.0 && r[b] + d[b] > 1.0) t = fmin(t, (1.0 - r[b]) / d[b]);
            if (d[b] < 0.0 && r[b] + d[b] < -1.0) t = fmin(t, (-1.0 - r[b]) / d[b]);
        }
        double rn[3] = { 0, 0, 0 }, s[3] = { 0, 0, 0 };
        for (int b = 0; b < dim; ++b) {
            rn[b] = r[b] + t * d[b];
            if (rn[b] > 1.0) rn[b] = 1.0;
            if (rn[b] < -1.0) rn[b] = -1.0;
            /* land exactly on the bound the step was cut at */
            if (t < 1.0 && d[b] > 0.0 && (1.0 - r[b]) / d[b] == t) rn[b] = 1.0;
            if (t < 1.0 && d[b] < 0.0 && (-1.0 - r[b]) / d[b] == t) rn[b] = -1.0;
            s[b] = rn[b] - r[b];
        }
        double sn = fmax(fabs(s[0]), fmax(fabs(s[1]), fabs(s[2])));
        if (sn == 0.0) break;
        /* predicted decrease of the Gauss-Newton model */
        double mf[3];
        for (int a = 0; a < dim; ++a) {
            mf[a] = f[a];
            for (int b = 0; b < dim; ++b) mf[a] += J[3 * a + b] * s[b];
        }
        double pred = phi - 0.5 * sumsq(dim, mf);
        double xn[3], Jn[9], fn[3] = { 0, 0, 0 };
        or_map_elem(el, rn, xn, Jn);
        for (int a = 0; a < dim; ++a) fn[a] = xn[a] - xs[a];
        double phin = 0.5 * sumsq(dim, fn);
        double dec = phi - phin;
        if (sn <= 1e-13) {                        /* converged in r */
            if (phin <= phi) { memcpy(r, rn, sizeof rn); phi = phin; }
            break;
        }
        if (dec > 0.0) {
            memcpy(r, rn, sizeof rn);
            memcpy(J, Jn, sizeof Jn);
            memcpy(f, fn, sizeof fn);
            phi = phin;
            double ratio = pred > 0.0 ? dec / pred : 0.0;
            if (ratio > 0.75 && sn >= 0.99 * rho) rho = fmin(2.0 * rho, 2.0);
            else if (ratio < 0.25) rho = 0.25 * sn;
        } else {
            rho = 0.25 * sn;
            if (rho < 1e-15) break;
        }
    }
    return sqrt(2.0 * phi);
}

/* ------------------------------------------------------------------------ */
/* Per-element helpers                                                      */
/* ------------------------------------------------------------------------ */

static void node_box(const double *const X[3], int d, int n3, double lo[3], double hi[3])
{
    lo[2] = hi[2] = 0.0;
    for (int a = 0; a < d; ++a) {
        double mn = X[a][0], mx = X[a][0];
        for (int q = 1; q < n3; ++q) {
            if (X[a][q] < mn) mn = X[a][q];
            if (X[a][q] > mx) mx = X[a][q];
        }
        lo[a] = mn;
        hi[a] = mx;
    }
}

static double diag3(const double lo[3], const double hi[3])
{
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Nearest mapped GLL node (Sec. 2.1: initial guess = closest point of the
   mapped GLL mesh); ties go to the lowest node index.  `skip` excludes the
   first `nskip` ranks so that restarts can take the next-nearest nodes. */
static int nearest_node(const or_elem *el, const double xs[3], int rank_wanted)
{
    int n3 = el->d == 2 ? el->n * el->n : el->n * el->n * el->n;
    /* select the rank_wanted-th smallest distance (0 = nearest) by repeated
       minimum search; plain and slow on purpose */
    double last = -1.0;
    int last_idx = -1, best = 0;
    for (int k = 0; k <= rank_wanted; ++k) {
        double bd = INFINITY;
        int bi = -1;
        for (int q = 0; q < n3; ++q) {
            double dx = el->X[0][q] - xs[0], dy = el->X[1][q] - xs[1];
            double d2 = dx * dx + dy * dy;
            if (el->d == 3) {
                double dz = el->X[2][q] - xs[2];
                d2 = d2 + dz * dz;
            }
            /* strictly after (last, last_idx) in (distance, index) order */
            int after = (d2 > last) || (d2 == last && q > last_idx);
            if (!after) continue;
            if (d2 < bd) { bd = d2; bi = q; }
        }
        if (bi < 0) return -1;
        last = bd;
        last_idx = bi;
        best = bi;
    }
    return best;
}

static void node_rst(const or_elem *el, int q, double r[3])
{
    int n = el->n;
    r[0] = el->xg[q % n];
    r[1] = el->xg[(q / n) % n];
    r[2] = el->d == 3 ? el->xg[q / (n * n)] : 0.0;
}

static double interp_elem(int N, int dim, const double *xg, const double *f, const double r[3])
{
    int n = N + 1;
    double h[3][OR_NMAX];
    for (int d = 0; d < dim; ++d) or_lagrange(N, xg, r[d], h[d], NULL);
    double v = 0.0;
    if (dim == 2) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) v += f[i + n * j] * h[0][i] * h[1][j];
        return v;
    }
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                v += f[i + n * (j + n * k)] * h[0][i] * h[1][j] * h[2][k];
    return v;
}

/* ------------------------------------------------------------------------ */
/* findpts by brute force                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double tol_accept;     /* INSIDE if residual <= tol_accept * h_e          */
    double tol_border;     /* BORDER if residual <= tol_border * h_e          */
    double tie_band;       /* owner / border ties: band = tie_band * L        */
    int max_newton;        /* Newton iteration cap                            */
    int n_restarts;        /* extra Newton starts from next-nearest nodes     */
    int prefilter;         /* 1: skip elements whose node box, grown by 25% of
                              its extent per side, misses x*                  */
} or_params;

/* Returns 0, or -1 for bad arguments (dim not 2 or 3, N out of range). */
int64_t or_find_d(int dim, int N, int64_t E, const double *coords, const int32_t *sub,
                  const double *dist, int64_t P, const double *pts, const int32_t *qsess,
                  const or_params *prm, int32_t *code, int32_t *osub, int32_t *oelem,
                  double *rst, double *dist2)
{
    double xg[OR_NMAX];
    if ((dim != 2 && dim != 3) || or_gll(N, xg, NULL)) return -1;
    int n = N + 1, n3 = dim == 2 ? n * n : n * n * n;
    double *elo = (double *)malloc(sizeof(double) * 3 * E);
    double *ehi = (double *)malloc(sizeof(double) * 3 * E);
    double *he = (double *)malloc(sizeof(double) * E);
    double glo[3] = { INFINITY, INFINITY, INFINITY }, ghi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int64_t e = 0; e < E; ++e) {
        const double *X[3] = { coords + e * n3, coords + (E + e) * n3, dim == 3 ? coords + (2 * E + e) * n3 : NULL };
        node_box(X, dim, n3, elo + 3 * e, ehi + 3 * e);
        he[e] = diag3(elo + 3 * e, ehi + 3 * e);
        for (int a = 0; a < 3; ++a) {
            if (elo[3 * e + a] < glo[a]) glo[a] = elo[3 * e + a];
            if (ehi[3 * e + a] > ghi[a]) ghi[a] = ehi[3 * e + a];
        }
    }
    double L = diag3(glo, ghi);
    double band = prm->tie_band * L;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
        double xs[3] = { pts[p], pts[P + p], dim == 3 ? pts[2 * P + p] : 0.0 };
        int32_t tag = qsess ? qsess[p] : -1;
        code[p] = OR_NOT_FOUND;
        osub[p] = -1;
        oelem[p] = -1;
        for (int a = 0; a < dim; ++a) rst[a * P + p] = 0.0;
        dist2[p] = INFINITY;
        if (!isfinite(xs[0]) || !isfinite(xs[1]) || !isfinite(xs[2])) continue;

        /* per-subdomain best INSIDE element (lowest id) -- subdomain ids are
           small non-negative integers; keep a short list */
        enum { MAXS = 64 };
        int64_t in_e[MAXS];
        int32_t in_s[MAXS];
        double in_r[MAXS][3], in_d[MAXS];
        int nin = 0;
        /* border bookkeeping */
        double bmin = INFINITY;
        int64_t b_e = -1;
        double b_r[3] = { 0, 0, 0 }, b_d = INFINITY;
        /* all border-eligible candidates, to apply the band rule at the end */
        int64_t *bc_e = NULL;
        double *bc_d = NULL, *bc_r = NULL;
        int nbc = 0, cap = 0;

        for (int64_t e = 0; e < E; ++e) {
            if (tag >= 0 && sub[e] == tag) continue;
            const double *lo = elo + 3 * e, *hi = ehi + 3 * e;
            if (prm->prefilter) {
                int out = 0;
                for (int a = 0; a < dim; ++a) {
                    double g = 0.25 * (hi[a] - lo[a]) + prm->tol_border * he[e];
                    if (xs[a] < lo[a] - g || xs[a] > hi[a] + g) out = 1;
                }
                if (out) continue;
            }
            or_elem el = { N, n, dim, xg, { coords + e * n3, coords + (E + e) * n3,
                                            dim == 3 ? coords + (2 * E + e) * n3 : NULL } };
            double r[3], best_r[3] = { 0, 0, 0 };
            double res = INFINITY;
            for (int k = 0; k <= prm->n_restarts && k < n3; ++k) {
                int q = nearest_node(&el, xs, k);
                if (q < 0) break;
                node_rst(&el, q, r);
                double rr = or_newton(&el, xs, r, prm->max_newton);
                if (rr < res) { res = rr; memcpy(best_r, r, sizeof r); }
                if (res <= prm->tol_accept * he[e]) break;
            }
            if (res <= prm->tol_accept * he[e]) {
                int s;
                for (s = 0; s < nin; ++s) if (in_s[s] == sub[e]) break;
                if (s == nin && nin < MAXS) {
                    in_s[nin] = sub[e]; in_e[nin] = e;
                    memcpy(in_r[nin], best_r, sizeof best_r); in_d[nin] = res; ++nin;
                }
                /* elements visited in increasing id: the first INSIDE element
                   of a subdomain is its lowest id; later ones are ignored */
            } else if (res <= prm->tol_border * he[e]) {
                if (nbc == cap) {
                    cap = cap ? 2 * cap : 8;
                    bc_e = (int64_t *)realloc(bc_e, sizeof(int64_t) * cap);
                    bc_d = (double *)realloc(bc_d, sizeof(double) * cap);
                    bc_r = (double *)realloc(bc_r, sizeof(double) * 3 * cap);
                }
                bc_e[nbc] = e; bc_d[nbc] = res; memcpy(bc_r + 3 * nbc, best_r, sizeof best_r); ++nbc;
                if (res < bmin) bmin = res;
            }
        }

        if (nin > 0) {
            int w = 0;
            if (nin > 1) {
                /* owner = argmax_k delta^k(x*), delta^k interpolated from the
                   nodal distance field at that subdomain's (e, r); within the
                   tie band the lower subdomain id wins (Sec. 2.1) */
                double dl[MAXS], dmax = -INFINITY;
                for (int s = 0; s < nin; ++s) {
                    dl[s] = dist ? interp_elem(N, dim, xg, dist + in_e[s] * n3, in_r[s]) : 0.0;
                    if (dl[s] > dmax) dmax = dl[s];
                }
                w = -1;
                for (int s = 0; s < nin; ++s)
                    if (dl[s] >= dmax - band && (w < 0 || in_s[s] < in_s[w])) w = s;
            }
            code[p] = OR_INSIDE;
            osub[p] = in_s[w];
            oelem[p] = (int32_t)in_e[w];
            for (int a = 0; a < dim; ++a) rst[a * P + p] = in_r[w][a];
            dist2[p] = in_d[w] * in_d[w];
        } else if (nbc > 0) {
            for (int c = 0; c < nbc; ++c)
                if (bc_d[c] <= bmin + band && (b_e < 0 || bc_e[c] < b_e)) {
                    b_e = bc_e[c]; b_d = bc_d[c]; memcpy(b_r, bc_r + 3 * c, sizeof b_r);
                }
            code[p] = OR_BORDER;
            osub[p] = sub[b_e];
            oelem[p] = (int32_t)b_e;
            for (int a = 0; a < dim; ++a) rst[a * P + p] = b_r[a];
            dist2[p] = b_d * b_d;
        }
        free(bc_e); free(bc_d); free(bc_r);
    }
    free(elo); free(ehi); free(he);
    return 0;
}

int64_t or_find(int N, int64_t E, const double *coords, const int32_t *sub,
                const double *dist, int64_t P, const double *pts, const int32_t *qsess,
                const or_params *prm, int32_t *code, int32_t *osub, int32_t *oelem,
                double *rst, double *dist2)
{
    return or_find_d(3, N, E, coords, sub, dist, P, pts, qsess, prm, code, osub, oelem, rst, dist2);
}

/* ------------------------------------------------------------------------ */
/* findpts_eval: full triple sum                                            */
/* ------------------------------------------------------------------------ */

/* out[f][p] = sum_ijk F[f][e][ijk] h_i(r) h_j(s) h_k(t) at (elem[p], rst[.][p]);
   NaN where code is NOT_FOUND (Sec. 2.1, findpts_eval). */
void or_eval_d(int dim, int N, int64_t E, int64_t P, const int32_t *code, const int32_t *elem,
               const double *rst, int F, const double *fields, double *out)
{
    double xg[OR_NMAX];
    or_gll(N, xg, NULL);
    int n = N + 1, n3 = dim == 2 ? n * n : n * n * n;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        double r[3] = { rst[p], rst[P + p], dim == 3 ? rst[2 * P + p] : 0.0 };
        for (int f = 0; f < F; ++f) {
            if (code[p] == OR_NOT_FOUND || elem[p] < 0) { out[f * P + p] = NAN; continue; }
            out[f * P + p] = interp_elem(N, dim, xg, fields + ((int64_t)f * E + elem[p]) * n3, r);
        }
    }
}

void or_eval(int N, int64_t E, int64_t P, const int32_t *code, const int32_t *elem,
             const double *rst, int F, const double *fields, double *out)
{
    or_eval_d(3, N, E, P, code, elem, rst, F, fields, out);
}

/* ------------------------------------------------------------------------ */
/* Default nodal distance field D^k                                         */
/* ------------------------------------------------------------------------ */

/* Local node index of (a,b) on face f of the reference cube:
   f = 0,1: r = -1,+1 (i = 0,N), (j,k) = (a,b); f = 2,3: s = -1,+1, (i,k) = (a,b);
   f = 4,5: t = -1,+1, (i,j) = (a,b). */
static int face_node(int n, int f, int a, int b)
{
    int N = n - 1, end = (f % 2) ? N : 0;
    switch (f / 2) {
    case 0: return end + n * (a + n * b);
    case 1: return a + n * (end + n * b);
    default: return a + n * (b + n * end);
    }
}

static int pt_less(const double *p, const double *q)
{
    for (int a = 0; a < 3; ++a) {
        if (p[a] < q[a]) return 1;
        if (p[a] > q[a]) return 0;
    }
    return 0;
}

/* the four corner points of face f of element e, sorted lexicographically */
static void face_corners(const double *coords, int64_t E, int n, int64_t e, int f, double c[4][3])
{
    int N = n - 1, n3 = n * n * n;
    int ab[4][2] = { { 0, 0 }, { N, 0 }, { 0, N }, { N, N } };
    for (int q = 0; q < 4; ++q) {
        int idx = face_node(n, f, ab[q][0], ab[q][1]);
        for (int a = 0; a < 3; ++a) c[q][a] = coords[(a * E + e) * n3 + idx];
    }
    for (int i = 1; i < 4; ++i)
        for (int j = i; j > 0 && pt_less(c[j], c[j - 1]); --j)
            for (int a = 0; a < 3; ++a) { double t = c[j][a]; c[j][a] = c[j - 1][a]; c[j - 1][a] = t; }
}

/* D^k(node) = min Euclidean distance from the node to the GLL nodes of the
   boundary faces of its own subdomain, where a boundary face is an element
   face whose four corners match no face of another element of the same
   subdomain (distance to the subdomain boundary, Sec. 2.1).  Brute force:
   O(faces^2) matching and O(nodes x boundary nodes) distances. */
int or_dist_default(int N, int64_t E, const double *coords, const int32_t *sub, double *D)
{
    int n = N + 1, n2 = n * n, n3 = n2 * n;
    int64_t F = 6 * E;
    char *bnd = (char *)malloc((size_t)F);
    double (*cor)[4][3] = malloc(sizeof(double[4][3]) * (size_t)F);
    for (int64_t e = 0; e < E; ++e)
        for (int f = 0; f < 6; ++f) face_corners(coords, E, n, e, f, cor[6 * e + f]);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t a = 0; a < F; ++a) {
        int shared = 0;
        for (int64_t b = 0; b < F && !shared; ++b) {
            if (b / 6 == a / 6 || sub[b / 6] != sub[a / 6]) continue;
            if (memcmp(cor[a], cor[b], sizeof(double[4][3])) == 0) shared = 1;
        }
        bnd[a] = !shared;
    }
    /* gather boundary-face nodes per element owner subdomain */
    int64_t nb = 0;
    for (int64_t a = 0; a < F; ++a) nb += bnd[a] ? n2 : 0;
    double *bx = (double *)malloc(sizeof(double) * 3 * (nb ? nb : 1));
    int32_t *bs = (int32_t *)malloc(sizeof(int32_t) * (nb ? nb : 1));
    int64_t m = 0;
    for (int64_t a = 0; a < F; ++a) {
        if (!bnd[a]) continue;
        int64_t e = a / 6;
        int f = (int)(a % 6);
        for (int bb = 0; bb < n; ++bb)
            for (int aa = 0; aa < n; ++aa) {
                int idx = face_node(n, f, aa, bb);
                for (int c = 0; c < 3; ++c) bx[3 * m + c] = coords[(c * E + e) * n3 + idx];
                bs[m] = sub[e];
                ++m;
            }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e) {
        for (int q = 0; q < n3; ++q) {
            double x = coords[e * n3 + q], y = coords[(E + e) * n3 + q], z = coords[(2 * E + e) * n3 + q];
            double best = INFINITY;
            for (int64_t b = 0; b < nb; ++b) {
                if (bs[b] != sub[e]) continue;
                double dx = x - bx[3 * b], dy = y - bx[3 * b + 1], dz = z - bx[3 * b + 2];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < best) best = d2;
            }
            D[e * n3 + q] = sqrt(best);
        }
    }
    free(bnd); free(cor); free(bx); free(bs);
    return 0;
}

/* The same field on a 2D quadrilateral mesh (coords [2][E][n^2]): boundary
   edges are element edges whose two end points match no edge of another
   element of the same subdomain; edge f = 0,1 is r = -1,+1 (nodes i = 0,N,
   j = 0..N), f = 2,3 is s = -1,+1. */
static int edge_node(int n, int f, int a)
{
    int end = (f % 2) ? n - 1 : 0;
    return f / 2 == 0 ? end + n * a : a + n * end;
}

int or_dist_default_2d(int N, int64_t E, const double *coords, const int32_t *sub, double *D)
{
    int n = N + 1, n2 = n * n;
    int64_t F = 4 * E;
    char *bnd = (char *)malloc((size_t)F);
    double (*cor)[2][2] = malloc(sizeof(double[2][2]) * (size_t)F);
    for (int64_t e = 0; e < E; ++e)
        for (int f = 0; f < 4; ++f) {
            double *c0 = cor[4 * e + f][0], *c1 = cor[4 * e + f][1];
            int i0 = edge_node(n, f, 0), i1 = edge_node(n, f, N);
            for (int a = 0; a < 2; ++a) {
                c0[a] = coords[(a * E + e) * n2 + i0];
                c1[a] = coords[(a * E + e) * n2 + i1];
            }
            /* sort the two end points lexicographically */
            if (c1[0] < c0[0] || (c1[0] == c0[0] && c1[1] < c0[1]))
                for (int a = 0; a < 2; ++a) { double t = c0[a]; c0[a] = c1[a]; c1[a] = t; }
        }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t a = 0; a < F; ++a) {
        int shared = 0;
        for (int64_t b = 0; b < F && !shared; ++b) {
            if (b / 4 == a / 4 || sub[b / 4] != sub[a / 4]) continue;
            if (memcmp(cor[a], cor[b], sizeof(double[2][2])) == 0) shared = 1;
        }
        bnd[a] = !shared;
    }
    int64_t nb = 0;
    for (int64_t a = 0; a < F; ++a) nb += bnd[a] ? n : 0;
    double *bx = (double *)malloc(sizeof(double) * 2 * (nb ? nb : 1));
    int32_t *bs = (int32_t *)malloc(sizeof(int32_t) * (nb ? nb : 1));
    int64_t m = 0;
    for (int64_t a = 0; a < F; ++a) {
        if (!bnd[a]) continue;
        int64_t e = a / 4;
        for (int q = 0; q < n; ++q) {
            int idx = edge_node(n, (int)(a % 4), q);
            bx[2 * m] = coords[e * n2 + idx];
            bx[2 * m + 1] = coords[(E + e) * n2 + idx];
            bs[m] = sub[e];
            ++m;
        }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e) {
        for (int q = 0; q < n2; ++q) {
            double x = coords[e * n2 + q], y = coords[(E + e) * n2 + q];
            double best = INFINITY;
            for (int64_t b = 0; b < nb; ++b) {
                if (bs[b] != sub[e]) continue;
                double dx = x - bx[2 * b], dy = y - bx[2 * b + 1];
                double d2 = dx * dx + dy * dy;
                if (d2 < best) best = d2;
            }
            D[e * n2 + q] = sqrt(best);
        }
    }
    free(bnd); free(cor); free(bx); free(bs);
    return 0;
}

/* number of OpenMP threads the oracle will use */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* number of OpenMP threads the oracle's later loops use (n >= 1; for timing
   it on one core beside all of them) */
void or_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Mass-flux correction on a subdomain boundary (Sec. 2.2, Eqs. consv1,     */
/* corr, consv2)                                                            */
/* ------------------------------------------------------------------------ */

/* Boundary-face quadrature.  kind[6E]: 0 = not used, 1 = boundary face with
   prescribed (Dirichlet) data, 2 = interface face (interpolated data).  The
   marked faces are listed in (element, face) order; face f's node (a,b) is
   numbered as in face_node().  For every listed node: position x, outward
   unit normal nrm and quadrature weight dA = w_a w_b |t_1 x t_2| (GLL
   weights, tangents t along the two face directions, from the derivative
   of the Lagrange interpolant of the node positions).  Outward: the face at
   the +1 end of a reference direction points along +(t_1 x t_2) for the
   cyclic pair (t_1, t_2) of the other two directions, times the sign of the
   element's Jacobian determinant at its centre.  Returns the number of
   listed nodes (arrays must hold 6*E*n^2 entries). */
int64_t or_bfaces(int N, int64_t E, const double *coords, const int8_t *kind, double *x, double *nrm,
                  double *dA, int8_t *nkind)
{
    double xg[OR_NMAX], wg[OR_NMAX];
    if (or_gll(N, xg, wg)) return -1;
    int n = N + 1, n3 = n * n * n;
    /* derivative of each Lagrange basis function at each GLL node */
    double Dm[OR_NMAX][OR_NMAX];
    for (int a = 0; a < n; ++a) {
        double h[OR_NMAX], dh[OR_NMAX];
        or_lagrange(N, xg, xg[a], h, dh);
        for (int i = 0; i < n; ++i) Dm[a][i] = dh[i];
    }
    int64_t m = 0;
    for (int64_t e = 0; e < E; ++e) {
        const double *X[3] = { coords + e * n3, coords + (E + e) * n3, coords + (2 * E + e) * n3 };
        /* handedness: sign of det J at the element centre */
        or_elem el = { N, n, 3, xg, { X[0], X[1], X[2] } };
        double r0[3] = { 0, 0, 0 }, xc[3], Jc[9];
        or_map_elem(&el, r0, xc, Jc);
        double det = Jc[0] * (Jc[4] * Jc[8] - Jc[5] * Jc[7]) - Jc[1] * (Jc[3] * Jc[8] - Jc[5] * Jc[6]) +
                     Jc[2] * (Jc[3] * Jc[7] - Jc[4] * Jc[6]);
        double hand = det < 0 ? -1.0 : 1.0;
        for (int f = 0; f < 6; ++f) {
            if (!kind[6 * e + f]) continue;
            int ax = f / 2;
            double sgn = (f % 2 ? 1.0 : -1.0) * hand;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    double t1[3], t2[3];
                    for (int c = 0; c < 3; ++c) {
                        double s1 = 0.0, s2 = 0.0;
                        for (int q = 0; q < n; ++q) {
                            /* t1 along the first face variable, t2 along the second */
                            s1 += Dm[a][q] * X[c][face_node(n, f, q, b)];
                            s2 += Dm[b][q] * X[c][face_node(n, f, a, q)];
                        }
                        t1[c] = s1;
                        t2[c] = s2;
                    }
                    /* face variables: ax 0 -> (s,t), ax 1 -> (r,t), ax 2 -> (r,s);
                       cyclic normal: ax 0: s x t, ax 1: t x r = -(r x t), ax 2: r x s */
                    double nv[3] = { t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                                     t1[0] * t2[1] - t1[1] * t2[0] };
                    double o = (ax == 1 ? -1.0 : 1.0) * sgn;
                    double len = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                    int idx = face_node(n, f, a, b);
                    for (int c = 0; c < 3; ++c) {
                        x[3 * m + c] = X[c][idx];
                        nrm[3 * m + c] = o * nv[c] / len;
                    }
                    dA[m] = wg[a] * wg[b] * len;
                    nkind[m] = kind[6 * e + f];
                    ++m;
                }
        }
    }
    return m;
}

/* gamma = -(sum over all listed nodes of u.n dA) / (sum over interface nodes
   of n.n dA) and u_out = u + gamma n on interface nodes, u elsewhere
   (Eq. consv2, Eq. corr).  u, u_out are [M][3]. */
void or_flux_correct(int64_t M, const double *u, const double *nrm, const double *dA, const int8_t *nkind,
                     double *u_out, double *gamma, double *flux)
{
    double fl = 0.0, area = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        double un = u[3 * m] * nrm[3 * m] + u[3 * m + 1] * nrm[3 * m + 1] + u[3 * m + 2] * nrm[3 * m + 2];
        fl += un * dA[m];
        if (nkind[m] == 2)
            area += (nrm[3 * m] * nrm[3 * m] + nrm[3 * m + 1] * nrm[3 * m + 1] + nrm[3 * m + 2] * nrm[3 * m + 2]) * dA[m];
    }
    double g = area > 0.0 ? -fl / area : 0.0;
    for (int64_t m = 0; m < M; ++m)
        for (int c = 0; c < 3; ++c) u_out[3 * m + c] = u[3 * m + c] + (nkind[m] == 2 ? g * nrm[3 * m + c] : 0.0);
    *gamma = g;
    if (flux) *flux = fl;
}
